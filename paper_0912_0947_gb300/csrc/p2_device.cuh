// p2_device.cuh -- device routines of the paper's own layout (Sections VI
// and VII), shared by the single-image kernels (paper2.cu) and the
// persistent batched kernels (batched.cu).
//
// Row r of plane `plane` is A_r[x] = cover[(r*W + x)*channels + plane].  With
// Q = floor(W/4) (Section VI step 5: 4*|B| <= |A|), rows take Q message bytes
// each until fewer than Q remain (Section VII step 4): rows 0..R-2 take Q,
// row R-1 takes L_last = N - (R-1)*Q.  Block i of the paper's launch writes
// bit pair i of B[j] to A_r[L_r*i + j] (Section VI step 7); extraction ORs the
// pairs back (Section VII step 6).
//
// Work units:
//   unit  16 consecutive pixels of a row = CH 16-byte vectors (rows of whole
//         vectors, CH in {1,3,4}); pixel t keeps its plane byte at unit byte
//         t*CH + PLANE, a compile-time position.  One-pass out-of-place
//         embedding (2C + N bytes).
//   run   16 consecutive message bytes of a row: extraction reads the four
//         units at columns i*L + j0 and ORs their pairs.
//   row   thread j of a row handles B[r*Q + j] and its four plane bytes (any
//         channel count; in place; after a copy out of place).
#pragma once

#include "async_copy.cuh"
#include "internal.cuh"

namespace stego {
namespace p2 {

struct View {
    const uint8_t *src; // cover (embed) or stego (extract)
    uint8_t *dst;       // stego (embed)
    const uint8_t *msg_in;
    uint8_t *msg_out;
    uint64_t N;
    uint32_t W, H, channels, plane;
    uint32_t Q;      // bytes per full row, floor(W/4)
    uint32_t R;      // rows that carry data
    uint32_t L_last; // bytes in row R-1
    uint32_t pad;
};

__host__ __device__ inline View make_view(const uint8_t *src, uint8_t *dst, uint32_t W,
                                          uint32_t H, uint32_t channels, uint32_t plane,
                                          const uint8_t *msg_in, uint8_t *msg_out, uint64_t N)
{
    View v;
    v.src = src;
    v.dst = dst;
    v.msg_in = msg_in;
    v.msg_out = msg_out;
    v.N = N;
    v.W = W;
    v.H = H;
    v.channels = channels;
    v.plane = plane;
    v.Q = W / 4u;
    v.R = v.Q ? (uint32_t)((N + v.Q - 1) / v.Q) : 0u;
    v.L_last = v.R ? (uint32_t)(N - (uint64_t)(v.R - 1) * v.Q) : 0u;
    v.pad = 0;
    return v;
}

__device__ __forceinline__ uint32_t row_len(const View &a, uint32_t r)
{
    return r + 1 < a.R ? a.Q : (r + 1 == a.R ? a.L_last : 0u);
}

// Quarter of a carrying column (block i of the paper): 0..3.
__device__ __forceinline__ uint32_t quarter(uint32_t col, uint32_t L)
{
    return (col >= L) + (col >= 2 * L) + (col >= 3 * L);
}

// Byte B (compile-time) of a unit of CH vectors, as a reference to its word.
template <int CH, int B>
__device__ __forceinline__ uint32_t &unit_word(uint4 (&o)[CH])
{
    uint4 &v = o[B >> 4];
    constexpr int W = (B >> 2) & 3;
    return W == 0 ? v.x : W == 1 ? v.y : W == 2 ? v.z : v.w;
}

template <int CH, int B>
__device__ __forceinline__ uint32_t unit_word_c(const uint4 (&c)[CH])
{
    const uint4 &v = c[B >> 4];
    constexpr int W = (B >> 2) & 3;
    return W == 0 ? v.x : W == 1 ? v.y : W == 2 ? v.z : v.w;
}

// Compile-time plan of the byte moves between a unit's words and its pair
// words (pair t in byte t%4 of pair word t/4; pixel t's plane byte is unit
// byte t*CH + PLANE).
struct UnitPlan {
    int CH, PLANE;
    // pixel whose plane byte is unit byte b, or -1
    __host__ __device__ constexpr int pixel_at(int b) const
    {
        return (b >= PLANE && (b - PLANE) % CH == 0 && (b - PLANE) / CH < 16) ? (b - PLANE) / CH
                                                                             : -1;
    }
    // unit word WD: mask of its plane pairs, and the first and last pair
    // words it takes pairs from
    __host__ __device__ constexpr uint32_t put_mask(int WD) const
    {
        uint32_t m = 0;
        for (int b = 0; b < 4; ++b)
            if (pixel_at(4 * WD + b) >= 0)
                m |= 3u << (8 * b);
        return m;
    }
    __host__ __device__ constexpr int put_qa(int WD) const
    {
        for (int b = 0; b < 4; ++b)
            if (pixel_at(4 * WD + b) >= 0)
                return pixel_at(4 * WD + b) >> 2;
        return 0;
    }
    __host__ __device__ constexpr int put_qb(int WD) const
    {
        for (int b = 3; b >= 0; --b)
            if (pixel_at(4 * WD + b) >= 0)
                return pixel_at(4 * WD + b) >> 2;
        return 0;
    }
    // byte_perm selector placing the pairs of unit word WD from pair words
    // qa (selector 0-3) and qb (4-7); other bytes are masked off later
    __host__ __device__ constexpr uint32_t put_sel(int WD) const
    {
        uint32_t s = 0;
        for (int b = 0; b < 4; ++b) {
            const int t = pixel_at(4 * WD + b);
            const uint32_t d = t < 0 ? 0u : (uint32_t)((t >> 2) == put_qa(WD) ? (t & 3) : 4 + (t & 3));
            s |= d << (4 * b);
        }
        return s;
    }
    // pair word Q, byte J: the unit word and byte holding pixel 4Q+J
    __host__ __device__ constexpr int src_word(int Q, int J) const { return ((4 * Q + J) * CH + PLANE) >> 2; }
    __host__ __device__ constexpr int src_byte(int Q, int J) const { return ((4 * Q + J) * CH + PLANE) & 3; }
    // the k-th distinct unit word pair word Q reads (k = 0..3), or -1
    __host__ __device__ constexpr int gather_src(int Q, int k) const
    {
        int n = 0;
        for (int j = 0; j < 4; ++j) {
            if (j > 0 && src_word(Q, j) == src_word(Q, j - 1))
                continue;
            if (n == k)
                return src_word(Q, j);
            ++n;
        }
        return -1;
    }
    // selector of the first gather step (distinct words 0 and 1) and of the
    // step adding distinct word k >= 2 to what is gathered so far
    __host__ __device__ constexpr uint32_t gather_sel0(int Q) const
    {
        uint32_t s = 0;
        const int w0 = gather_src(Q, 0), w1 = gather_src(Q, 1);
        for (int j = 0; j < 4; ++j) {
            const int w = src_word(Q, j);
            const uint32_t d = w == w0 ? (uint32_t)src_byte(Q, j)
                                       : (w == w1 ? 4u + src_byte(Q, j) : 0u);
            s |= d << (4 * j);
        }
        return s;
    }
    __host__ __device__ constexpr uint32_t gather_selk(int Q, int k) const
    {
        uint32_t s = 0;
        const int wk = gather_src(Q, k);
        for (int j = 0; j < 4; ++j) {
            const uint32_t d = src_word(Q, j) == wk ? 4u + src_byte(Q, j) : (uint32_t)j;
            s |= d << (4 * j);
        }
        return s;
    }
};

// Pairs P (pair t in the low two bits of byte t%4 of P[t/4]; the other
// bits are ignored) into the plane bytes of a unit: per unit word one
// byte_perm from at most two pair words and one masked merge.
template <int CH, int PLANE, int WD = 0>
__device__ __forceinline__ void put_unit(uint4 (&o)[CH], const uint32_t (&P)[4])
{
    if constexpr (WD < 4 * CH) {
        constexpr UnitPlan pl{CH, PLANE};
        constexpr uint32_t M = pl.put_mask(WD);
        if constexpr (M != 0) {
            constexpr int QA = pl.put_qa(WD), QB = pl.put_qb(WD);
            constexpr uint32_t SEL = pl.put_sel(WD);
            uint32_t &w = unit_word<CH, 4 * WD>(o);
            const uint32_t p = __byte_perm(P[QA], P[QB], SEL);
            w = (w & ~M) | (p & M);
        }
        put_unit<CH, PLANE, WD + 1>(o, P);
    }
}

// Plane bytes of pixels 4Q..4Q+3 of a unit as one word (byte j = pixel
// 4Q+j's whole plane byte): a chain of byte_perms over the unit words that
// hold them.
template <int CH, int PLANE, int Q>
__device__ __forceinline__ uint32_t gather_word(const uint4 (&c)[CH])
{
    constexpr UnitPlan pl{CH, PLANE};
    constexpr int W0 = pl.gather_src(Q, 0), W1 = pl.gather_src(Q, 1);
    constexpr int W2 = pl.gather_src(Q, 2), W3 = pl.gather_src(Q, 3);
    uint32_t g = __byte_perm(unit_word_c<CH, 4 * W0>(c),
                             unit_word_c<CH, 4 * (W1 < 0 ? W0 : W1)>(c), pl.gather_sel0(Q));
    if constexpr (W2 >= 0)
        g = __byte_perm(g, unit_word_c<CH, 4 * W2>(c), pl.gather_selk(Q, 2));
    if constexpr (W3 >= 0)
        g = __byte_perm(g, unit_word_c<CH, 4 * W3>(c), pl.gather_selk(Q, 3));
    return g;
}

// Plane bytes of a unit's 16 pixels as four words (byte t%4 of G[t/4] =
// pixel t's plane byte).
template <int CH, int PLANE>
__device__ __forceinline__ void get_unit(const uint4 (&c)[CH], uint32_t (&G)[4])
{
    if constexpr (CH == 1) {
        G[0] = c[0].x;
        G[1] = c[0].y;
        G[2] = c[0].z;
        G[3] = c[0].w;
    } else {
        G[0] = gather_word<CH, PLANE, 0>(c);
        G[1] = gather_word<CH, PLANE, 1>(c);
        G[2] = gather_word<CH, PLANE, 2>(c);
        G[3] = gather_word<CH, PLANE, 3>(c);
    }
}

// Pairs of a unit's plane bytes (their low two bits) into a SWAR pair array
// (pair t in byte t%4 of P[t/4]; P starts zeroed), one shift and mask per
// pixel: in the extraction this measured faster than the byte_perm gather.
template <int CH, int PLANE, int T = 0>
__device__ __forceinline__ void get_pairs(const uint4 (&c)[CH], uint32_t (&P)[4])
{
    if constexpr (T < 16) {
        constexpr int B = T * CH + PLANE, S = 8 * (B & 3);
        const uint32_t w = unit_word_c<CH, B & ~3>(c);
        P[T >> 2] |= ((w >> S) & 3u) << (8 * (T & 3));
        get_pairs<CH, PLANE, T + 1>(c, P);
    }
}

// Per-pixel path for a unit that crosses a quarter boundary or the end of
// the carrying columns: pixel T at column colf + T.
template <int CH, int PLANE, int T>
__device__ __forceinline__ void slow_unit(uint4 (&o)[CH], uint32_t colf, uint32_t L,
                                          const uint8_t *__restrict__ mrow)
{
    if constexpr (T < 16) {
        const uint32_t col = colf + T;
        if (col < 4 * L) {
            const uint32_t i = quarter(col, L);
            const uint32_t p = (__ldg(mrow + (col - i * L)) >> (2 * i)) & 3u;
            constexpr int B = T * CH + PLANE, S = 8 * (B & 3);
            uint32_t &w = unit_word<CH, B>(o);
            w = (w & ~(3u << S)) | (p << S);
        }
        slow_unit<CH, PLANE, T + 1>(o, colf, L, mrow);
    }
}

// Four 32-bit words of message bytes mp[0..15] (mp 4-byte aligned or not).
__device__ __forceinline__ void load16(const uint8_t *__restrict__ mp, uint32_t (&m)[4])
{
    if (((uintptr_t)mp & 15u) == 0) {
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(mp));
        m[0] = v.x;
        m[1] = v.y;
        m[2] = v.z;
        m[3] = v.w;
    } else if (((uintptr_t)mp & 3u) == 0) {
        const uint32_t *w = reinterpret_cast<const uint32_t *>(mp);
#pragma unroll
        for (int q = 0; q < 4; ++q)
            m[q] = __ldg(w + q);
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q)
            m[q] = (uint32_t)__ldg(mp + 4 * q) | ((uint32_t)__ldg(mp + 4 * q + 1) << 8) |
                   ((uint32_t)__ldg(mp + 4 * q + 2) << 16) | ((uint32_t)__ldg(mp + 4 * q + 3) << 24);
    }
}

// Changed plane bytes and squared error of a unit from its new and old
// plane bytes (byte t%4 of word t/4 = pixel t; only the low two bits can
// differ, the other bits are ignored), added to 32-bit per-unit counts.
__device__ __forceinline__ void plane_stats(const uint32_t (&Gn)[4], const uint32_t (&Go)[4],
                                            uint32_t &n, uint32_t &s)
{
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint32_t d = __vabsdiffu4(Gn[q] & 0x03030303u, Go[q] & 0x03030303u);
        n += __popc((d | (d >> 1)) & 0x01010101u);
        s = __dp4a(d, d, s);
    }
}

// (row, unit column) advanced by dr rows and dc < upr units.
__device__ __forceinline__ void rc_add(uint32_t &r, uint32_t &c, uint32_t dr, uint32_t dc,
                                       uint32_t upr)
{
    r += dr;
    c += dc;
    if (c >= upr) {
        c -= upr;
        ++r;
    }
}

// Units with carrying pixels, a prefix of the image's units: every unit of
// rows 0..R-2 (4Q = W when W is a multiple of 16) and the first
// ceil(L_last/4) of row R-1.
__device__ __forceinline__ uint32_t carrying_units(const View &a, uint32_t upr)
{
    return a.R ? (a.R - 1) * upr + (a.L_last + 3) / 4 : 0u;
}

constexpr int kStageWarps = 8; // units_embed_async runs in CTAs of at most 256 threads

// One pass over units k = k_first + i*step (+ u*blockDim.x, u < UT),
// k < k_end, of an image whose rows are whole units and whose buffers are
// 16-byte aligned, each thread on its own units: every load of an iteration
// (cover, then message) is issued before any arithmetic.  With one channel
// the lanes' single-vector units are consecutive (coalesced); with three or
// four a lane's unit lies 16*CH bytes from its neighbour's, which
// units_embed_async avoids and the batched kernels accept for their register
// budget.  Out of place every unit is written (units without carrying pixels
// are copied); in place (INPLACE) k_end is cut to the carrying units, each
// unit read and written back by the same thread.
template <int CH, int PLANE, bool STATS, int UT, bool INPLACE = false>
__device__ __forceinline__ void units_embed(const View &a, uint32_t k_first, uint32_t k_end,
                                            uint32_t step, unsigned long long &changed,
                                            unsigned long long &sse)
{
    const uint32_t upr = a.W / 16; // units per row
    if (upr == 0)
        return;
    const uint32_t carry = carrying_units(a, upr);
    if (INPLACE && k_end > carry)
        k_end = carry;
    const uint4 *__restrict__ src = reinterpret_cast<const uint4 *>(a.src);
    uint4 *dst = reinterpret_cast<uint4 *>(a.dst);
    // row and unit column of the thread's unit: with several units per thread
    // kept by additions (the strides blockDim.x and step in whole rows and
    // remaining units), with one unit divided out (fewer live registers)
    constexpr bool TRACK = UT > 1;
    uint32_t r0 = 0, u0 = 0, tr = 0, tc = 0, sr = 0, sc = 0;
    if constexpr (TRACK) {
        r0 = k_first / upr;
        u0 = k_first - r0 * upr;
        tr = blockDim.x / upr;
        tc = blockDim.x - tr * upr;
        sr = step / upr;
        sc = step - sr * upr;
    }
    for (uint32_t k0 = k_first; k0 < k_end; k0 += step) {
        uint4 c[UT][CH];
#pragma unroll
        for (int u = 0; u < UT; ++u) {
            const uint32_t k = k0 + u * blockDim.x;
            if (k < k_end) {
#pragma unroll
                for (int q = 0; q < CH; ++q)
                    c[u][q] = __ldcs(src + (uint64_t)k * CH + q);
            }
        }
        int mode[UT]; // 0: copy only, 1: one quarter (SWAR), 2: per pixel
        uint32_t colf[UT], L[UT], i0[UT], m[UT][4];
        const uint8_t *mrow[UT];
        uint32_t r = r0, uc = u0;
#pragma unroll
        for (int u = 0; u < UT; ++u) {
            const uint32_t k = k0 + u * blockDim.x;
            if constexpr (TRACK) {
                if (u > 0)
                    rc_add(r, uc, tr, tc, upr);
            } else {
                r = k / upr;
                uc = k - r * upr;
            }
            mode[u] = 0;
            if (k < k_end && k < carry) {
                colf[u] = 16u * uc;
                L[u] = row_len(a, r);
                mrow[u] = a.msg_in + (uint64_t)r * a.Q;
                i0[u] = quarter(colf[u], L[u]);
                if (colf[u] + 15 < 4 * L[u] && quarter(colf[u] + 15, L[u]) == i0[u]) {
                    mode[u] = 1;
                    load16(mrow[u] + (colf[u] - i0[u] * L[u]), m[u]);
                } else {
                    mode[u] = 2;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < UT; ++u) {
            const uint32_t k = k0 + u * blockDim.x;
            if (k >= k_end)
                continue;
            uint4(&o)[CH] = c[u]; // rewritten in registers
            uint32_t Gn[4], Go[4];
            if (STATS && mode[u])
                get_unit<CH, PLANE>(o, Go); // old plane bytes
            if (mode[u] == 1) {
                // pair of quarter i0 in the low two bits of each byte
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    Gn[q] = m[u][q] >> (2 * i0[u]);
                if constexpr (CH == 1) {
                    o[0].x = (o[0].x & 0xFCFCFCFCu) | (Gn[0] & 0x03030303u);
                    o[0].y = (o[0].y & 0xFCFCFCFCu) | (Gn[1] & 0x03030303u);
                    o[0].z = (o[0].z & 0xFCFCFCFCu) | (Gn[2] & 0x03030303u);
                    o[0].w = (o[0].w & 0xFCFCFCFCu) | (Gn[3] & 0x03030303u);
                } else {
                    put_unit<CH, PLANE>(o, Gn);
                }
            } else if (mode[u] == 2) {
                slow_unit<CH, PLANE, 0>(o, colf[u], L[u], mrow[u]);
                if (STATS)
                    get_unit<CH, PLANE>(o, Gn);
            }
            if (STATS && mode[u]) {
                uint32_t n = 0, sq = 0; // at most 16 pairs changed, 9 each
                plane_stats(Gn, Go, n, sq);
                changed += n;
                sse += sq;
            }
#pragma unroll
            for (int q = 0; q < CH; ++q)
                __stcs(dst + (uint64_t)k * CH + q, o[q]);
        }
        if constexpr (TRACK)
            rc_add(r0, u0, sr, sc, upr);
    }
}

// What one unit needs besides its cover vectors: how it is embedded (mode
// 0 copy only, 1 one quarter, 2 per pixel), its column, row length,
// quarter, message row and, in mode 1, its 16 message bytes.
struct UnitJob {
    uint32_t mode, colf, L, i0;
    const uint8_t *mrow;
    uint32_t m[4];
};

__device__ __forceinline__ void plan_unit(const View &a, uint32_t k, uint32_t k_end,
                                          uint32_t carry, uint32_t r, uint32_t uc, UnitJob &J)
{
    J.mode = 0;
    if (k < k_end && k < carry) {
        J.colf = 16u * uc;
        J.L = row_len(a, r);
        J.mrow = a.msg_in + (uint64_t)r * a.Q;
        J.i0 = quarter(J.colf, J.L);
        if (J.colf + 15 < 4 * J.L && quarter(J.colf + 15, J.L) == J.i0) {
            J.mode = 1;
            load16(J.mrow + (J.colf - J.i0 * J.L), J.m);
        } else {
            J.mode = 2;
        }
    }
}

// units_embed for CH > 1 with a two-stage copy pipeline per warp: while the
// warp embeds the units of one iteration from shared memory, the cover
// vectors of its next iteration are already on their way there
// (cp.async, memory order, coalesced) and the next units' message bytes on
// their way to registers.  Same arguments and results as units_embed; CTAs
// of at most 256 threads.
template <int CH, int PLANE, bool STATS, int UT, bool INPLACE = false>
__device__ __forceinline__ void units_embed_async(const View &a, uint32_t k_first,
                                                  uint32_t k_end, uint32_t step,
                                                  unsigned long long &changed,
                                                  unsigned long long &sse)
{
    static_assert(CH > 1, "one-channel units are single vectors, loaded coalesced as they are");
    const uint32_t upr = a.W / 16;
    if (upr == 0)
        return;
    const uint32_t carry = carrying_units(a, upr);
    if (INPLACE && k_end > carry)
        k_end = carry;
    const uint4 *__restrict__ src = reinterpret_cast<const uint4 *>(a.src);
    uint4 *dst = reinterpret_cast<uint4 *>(a.dst);
    const uint32_t lane = threadIdx.x & 31u;
    constexpr uint32_t SV = unit_stage_slots<CH>();
    constexpr uint32_t WS = 2 * UT * SV; // two stages per warp
    __shared__ uint4 stage[kStageWarps * WS];
    uint4 *const sw = stage + (threadIdx.x >> 5) * WS;
    const uint64_t vend = (uint64_t)k_end * CH;
    const uint32_t tr = blockDim.x / upr, tc = blockDim.x - tr * upr;
    const uint32_t sr = step / upr, sc = step - sr * upr;
    uint32_t r0 = k_first / upr, u0 = k_first - r0 * upr;

    // the warp's vectors of the iteration at lane 0's unit kb -> stage s
    auto issue = [&](uint32_t kb, uint32_t s) {
#pragma unroll
        for (int u = 0; u < UT; ++u) {
            const uint64_t v0 = (uint64_t)(kb + u * blockDim.x) * CH;
#pragma unroll
            for (int j = 0; j < CH; ++j)
                if (v0 + 32u * j + lane < vend)
                    cp_async16(sw + s * UT * SV + u * SV + unit_stage_slot<CH>(32u * j + lane),
                               src + v0 + 32u * j + lane);
        }
        cp_async_commit();
    };
    auto plan = [&](uint32_t k0, uint32_t r, uint32_t uc, UnitJob (&J)[UT]) {
#pragma unroll
        for (int u = 0; u < UT; ++u) {
            if (u > 0)
                rc_add(r, uc, tr, tc, upr);
            plan_unit(a, k0 + u * blockDim.x, k_end, carry, r, uc, J[u]);
        }
    };

    uint32_t k0 = k_first; // the lane's first unit; k0 - lane is the same for the warp
    if (k0 - lane >= k_end)
        return;
    UnitJob J[UT];
    issue(k0 - lane, 0);
    plan(k0, r0, u0, J);
    uint32_t s = 0;
    for (;;) {
        const uint32_t kn = k0 + step;
        const bool next = kn - lane < k_end; // kn < 2^32: units and steps stay below 2^31
        UnitJob Jn[UT];
        rc_add(r0, u0, sr, sc, upr);
        if (next) {
            issue(kn - lane, s ^ 1u);
            plan(kn, r0, u0, Jn);
            cp_async_wait<1>(); // this iteration's copies landed (the next may be pending)
        } else {
            cp_async_wait<0>();
        }
        __syncwarp(); // every lane's copies visible to the warp
        uint4 *const st = sw + s * UT * SV;
#pragma unroll
        for (int u = 0; u < UT; ++u) {
            const uint32_t k = k0 + u * blockDim.x;
            if (k >= k_end)
                continue;
            uint4 o[CH];
#pragma unroll
            for (int q = 0; q < CH; ++q)
                o[q] = st[u * SV + unit_stage_slot<CH>(CH * lane + q)];
            uint32_t Gn[4], Go[4];
            if (STATS && J[u].mode)
                get_unit<CH, PLANE>(o, Go);
            if (J[u].mode == 1) {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    Gn[q] = J[u].m[q] >> (2 * J[u].i0);
                put_unit<CH, PLANE>(o, Gn);
            } else if (J[u].mode == 2) {
                slow_unit<CH, PLANE, 0>(o, J[u].colf, J[u].L, J[u].mrow);
                if (STATS)
                    get_unit<CH, PLANE>(o, Gn);
            }
            if (STATS && J[u].mode) {
                uint32_t n = 0, sq = 0;
                plane_stats(Gn, Go, n, sq);
                changed += n;
                sse += sq;
            }
            if (J[u].mode) {
#pragma unroll
                for (int q = 0; q < CH; ++q)
                    st[u * SV + unit_stage_slot<CH>(CH * lane + q)] = o[q];
            }
        }
        __syncwarp(); // the rewritten units visible to the storing lanes
#pragma unroll
        for (int u = 0; u < UT; ++u) {
            const uint64_t v0 = (uint64_t)(k0 - lane + u * blockDim.x) * CH;
#pragma unroll
            for (int j = 0; j < CH; ++j)
                if (v0 + 32u * j + lane < vend)
                    __stcs(dst + v0 + 32u * j + lane, st[u * SV + unit_stage_slot<CH>(32u * j + lane)]);
        }
        if (!next)
            break;
        // stage s is refilled two iterations on, after this lane's reads of
        // its own memory-order slots above
#pragma unroll
        for (int u = 0; u < UT; ++u)
            J[u] = Jn[u];
        k0 = kn;
        s ^= 1u;
    }
}

// Scatter of carrying rows r = r_first + i*r_step < min(r_end, R): the
// calling CTA's threads split each row's L message bytes, four per thread in
// flight; each reads B[r*Q + j] once and rewrites its four plane bytes (from
// src into dst; src may equal dst).
template <bool STATS>
__device__ __forceinline__ void rows_embed(const View &a, uint32_t r_first, uint32_t r_end,
                                           uint32_t r_step, unsigned long long &changed,
                                           unsigned long long &sse)
{
    const uint32_t rend = r_end < a.R ? r_end : a.R;
    for (uint32_t r = r_first; r < rend; r += r_step) {
        const uint32_t L = row_len(a, r);
        const uint8_t *mrow = a.msg_in + (uint64_t)r * a.Q;
        const uint64_t prow = (uint64_t)r * a.W;
        const uint64_t qstride = (uint64_t)L * a.channels; // pair i at base(j) + i*qstride
        constexpr int U = 4;
        for (uint32_t j0 = threadIdx.x; j0 < L; j0 += blockDim.x * U) {
            uint32_t B[U], c[U][4];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint32_t j = j0 + u * blockDim.x;
                if (j >= L)
                    continue;
                B[u] = __ldg(mrow + j);
                const uint8_t *p = a.src + (prow + j) * a.channels + a.plane;
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    c[u][i] = p[i * qstride]; // plain load: src may equal dst (in place)
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint32_t j = j0 + u * blockDim.x;
                if (j >= L)
                    continue;
                uint8_t *p = a.dst + (prow + j) * a.channels + a.plane;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const uint32_t v = (c[u][i] & 0xFCu) | ((B[u] >> (2 * i)) & 3u);
                    p[i * qstride] = (uint8_t)v;
                    if (STATS) {
                        const uint32_t d = v > c[u][i] ? v - c[u][i] : c[u][i] - v;
                        changed += d != 0;
                        sse += d * d;
                    }
                }
            }
        }
    }
}

// Copy of whole rows [r0, r1) from src to dst by the calling CTA (16-byte
// vectors where src and dst agree modulo 16, bytes otherwise).
__device__ __forceinline__ void rows_copy(const View &a, uint32_t r0, uint32_t r1)
{
    const uint64_t rb = (uint64_t)a.W * a.channels;
    const uint64_t b0 = r0 * rb, b1 = r1 * rb;
    const uint8_t *s = a.src;
    uint8_t *d = a.dst;
    const uint32_t ms = (uint32_t)((uintptr_t)(s + b0) & 15u);
    if (ms == ((uintptr_t)(d + b0) & 15u)) {
        const uint64_t head = ms ? 16u - ms : 0u;
        const uint64_t vb = b0 + head < b1 ? b0 + head : b1;          // first vector byte
        const uint64_t ve = vb + ((b1 - vb) & ~15ull);                // end of whole vectors
        for (uint64_t k = b0 + threadIdx.x; k < vb; k += blockDim.x)
            d[k] = s[k];
        const uint4 *sv = reinterpret_cast<const uint4 *>(s + vb);
        uint4 *dv = reinterpret_cast<uint4 *>(d + vb);
        const uint64_t nv = (ve - vb) >> 4;
        for (uint64_t k = threadIdx.x; k < nv; k += blockDim.x)
            __stcs(dv + k, __ldcs(sv + k));
        for (uint64_t k = ve + threadIdx.x; k < b1; k += blockDim.x)
            d[k] = s[k];
    } else {
        for (uint64_t k = b0 + threadIdx.x; k < b1; k += blockDim.x)
            d[k] = s[k];
    }
}

// Extraction over runs k = k_first + i*step < k_end of 16 message bytes of a
// carrying row (rpr = ceil(Q/16) runs per row): the four units at columns
// i*L + j0 are read as vectors when every one is a whole 16-byte aligned
// unit, byte by byte otherwise.
template <int CH, int PLANE>
__device__ __forceinline__ void runs_extract(const View &a, uint64_t k_first, uint64_t k_end,
                                             uint64_t step)
{
    const uint32_t rpr = (a.Q + 15) / 16;
    for (uint64_t k = k_first; k < k_end; k += step) {
        const uint32_t r = (uint32_t)(k / rpr);
        const uint32_t j0 = 16u * (uint32_t)(k - (uint64_t)r * rpr);
        const uint32_t L = row_len(a, r);
        if (j0 >= L)
            continue;
        const uint64_t prow = (uint64_t)r * a.W;
        uint8_t *mp = a.msg_out + (uint64_t)r * a.Q + j0;
        // whole unit per quarter, and every quarter's unit 16-byte aligned:
        // the first one aligned and the quarter stride L*CH a multiple of 16
        const bool fast = j0 + 16 <= L && ((uint64_t)L * CH) % 16u == 0 &&
                          (((uintptr_t)(a.src + (prow + j0) * CH)) & 15u) == 0;
        if (fast) {
            uint4 c[4][CH];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const uint4 *u = reinterpret_cast<const uint4 *>(
                    a.src + (prow + (uint64_t)L * i + j0) * CH);
#pragma unroll
                for (int q = 0; q < CH; ++q)
                    c[i][q] = __ldcs(u + q);
            }
            uint32_t M[4] = {0u, 0u, 0u, 0u};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                uint32_t P[4] = {0u, 0u, 0u, 0u};
                if constexpr (CH == 1) {
                    P[0] = c[i][0].x & 0x03030303u;
                    P[1] = c[i][0].y & 0x03030303u;
                    P[2] = c[i][0].z & 0x03030303u;
                    P[3] = c[i][0].w & 0x03030303u;
                } else {
                    get_pairs<CH, PLANE>(c[i], P);
                }
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    M[q] |= P[q] << (2 * i);
            }
            if (((uintptr_t)mp & 15u) == 0) {
                *reinterpret_cast<uint4 *>(mp) = make_uint4(M[0], M[1], M[2], M[3]);
            } else {
#pragma unroll
                for (int t = 0; t < 16; ++t)
                    mp[t] = (uint8_t)(M[t >> 2] >> (8 * (t & 3)));
            }
        } else {
            const uint32_t n = L - j0 < 16u ? L - j0 : 16u;
            for (uint32_t t = 0; t < n; ++t) {
                uint32_t B = 0;
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    B |= (uint32_t)(a.src[(prow + (uint64_t)L * i + j0 + t) * CH + PLANE] & 3u)
                         << (2 * i);
                mp[t] = (uint8_t)B;
            }
        }
    }
}

// Extraction of carrying rows r = r_first + i*r_step < min(r_end, R), any
// channel count: the calling CTA's threads split each row's L bytes.
__device__ __forceinline__ void rows_extract(const View &a, uint32_t r_first, uint32_t r_end,
                                             uint32_t r_step)
{
    const uint32_t rend = r_end < a.R ? r_end : a.R;
    for (uint32_t r = r_first; r < rend; r += r_step) {
        const uint32_t L = row_len(a, r);
        uint8_t *mrow = a.msg_out + (uint64_t)r * a.Q;
        const uint64_t prow = (uint64_t)r * a.W;
        constexpr int U = 4;
        for (uint32_t j0 = threadIdx.x; j0 < L; j0 += blockDim.x * U) {
            uint32_t c[U][4];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint32_t j = j0 + u * blockDim.x;
                if (j >= L)
                    continue;
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    c[u][i] = __ldg(a.src + (prow + (uint64_t)L * i + j) * a.channels + a.plane);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint32_t j = j0 + u * blockDim.x;
                if (j >= L)
                    continue;
                uint32_t B = 0;
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    B |= (c[u][i] & 3u) << (2 * i);
                mrow[j] = (uint8_t)B;
            }
        }
    }
}

// Runtime (channels, plane) -> the templated run routine.
__device__ __forceinline__ void runs_extract_any(const View &a, uint64_t k_first, uint64_t k_end,
                                                 uint64_t step)
{
    switch (a.channels * 4 + a.plane) {
    case 4: runs_extract<1, 0>(a, k_first, k_end, step); break;
    case 12: runs_extract<3, 0>(a, k_first, k_end, step); break;
    case 13: runs_extract<3, 1>(a, k_first, k_end, step); break;
    case 14: runs_extract<3, 2>(a, k_first, k_end, step); break;
    case 16: runs_extract<4, 0>(a, k_first, k_end, step); break;
    case 17: runs_extract<4, 1>(a, k_first, k_end, step); break;
    case 18: runs_extract<4, 2>(a, k_first, k_end, step); break;
    case 19: runs_extract<4, 3>(a, k_first, k_end, step); break;
    default: break;
    }
}

// The layouts the unit and run routines handle.
__host__ __device__ inline bool unit_channels(uint32_t ch) { return ch == 1 || ch == 3 || ch == 4; }

} // namespace p2
} // namespace stego
