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

// Pair of pixel T (0..15) from a SWAR pair array (pair t in byte t%4 of
// word t/4) into the unit's plane byte.
template <int CH, int PLANE, int T>
__device__ __forceinline__ void put_unit(uint4 (&o)[CH], const uint32_t (&P)[4])
{
    if constexpr (T < 16) {
        constexpr int B = T * CH + PLANE, S = 8 * (B & 3);
        uint32_t &w = unit_word<CH, B>(o);
        const uint32_t p = (P[T >> 2] >> (8 * (T & 3))) & 3u;
        w = (w & ~(3u << S)) | (p << S);
        put_unit<CH, PLANE, T + 1>(o, P);
    }
}

// Plane-byte pairs of a unit (low two bits) into a SWAR pair array.
template <int CH, int PLANE, int T>
__device__ __forceinline__ void get_unit(const uint4 (&c)[CH], uint32_t (&P)[4])
{
    if constexpr (T < 16) {
        constexpr int B = T * CH + PLANE, S = 8 * (B & 3);
        const uint4 &v = c[B >> 4];
        constexpr int W = (B >> 2) & 3;
        const uint32_t w = W == 0 ? v.x : W == 1 ? v.y : W == 2 ? v.z : v.w;
        P[T >> 2] |= ((w >> S) & 3u) << (8 * (T & 3));
        get_unit<CH, PLANE, T + 1>(c, P);
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
    if (((uintptr_t)mp & 3u) == 0) {
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

// Changed bytes and squared error of two vectors that differ only in the
// low two bits of some bytes, added to 32-bit per-unit counts.
__device__ __forceinline__ void pair_stats(const uint4 &o, const uint4 &c, uint32_t &n,
                                           uint32_t &s)
{
    const uint32_t ow[4] = {o.x, o.y, o.z, o.w}, cw[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint32_t x = ow[q] ^ cw[q];
        n += __popc((x | (x >> 1)) & 0x01010101u);
        const uint32_t d = __vabsdiffu4(ow[q] & 0x03030303u, cw[q] & 0x03030303u);
        s = __dp4a(d, d, s);
    }
}

// One pass over units k = k_first + i*step (+ u*blockDim.x, u < UT),
// k < k_end, of an image whose rows are whole units and whose buffers are
// 16-byte aligned.  Out of place every unit is written (units without
// carrying pixels are copied) and each thread issues the cover loads of its
// UT units, then their message loads, before any arithmetic.  In place
// (INPLACE, k_end at most the units of the carrying rows) only units with
// carrying pixels are read and written back whole.
template <int CH, int PLANE, bool STATS, int UT, bool INPLACE = false>
__device__ __forceinline__ void units_embed(const View &a, uint32_t k_first, uint32_t k_end,
                                            uint32_t step, unsigned long long &changed,
                                            unsigned long long &sse)
{
    const uint32_t upr = a.W / 16; // units per row
    const uint32_t carry_units = upr * a.R;
    const uint4 *__restrict__ src = reinterpret_cast<const uint4 *>(a.src);
    uint4 *dst = reinterpret_cast<uint4 *>(a.dst);
    for (uint32_t k0 = k_first; k0 < k_end; k0 += step) {
        uint4 c[UT][CH];
        if constexpr (!INPLACE) {
#pragma unroll
            for (int u = 0; u < UT; ++u) {
                const uint32_t k = k0 + u * blockDim.x;
                if (k < k_end) {
#pragma unroll
                    for (int q = 0; q < CH; ++q)
                        c[u][q] = __ldcs(src + (uint64_t)k * CH + q);
                }
            }
        }
        int mode[UT]; // 0: copy only, 1: one quarter (SWAR), 2: per pixel
        uint32_t colf[UT], L[UT], i0[UT], m[UT][4];
        const uint8_t *mrow[UT];
#pragma unroll
        for (int u = 0; u < UT; ++u) {
            const uint32_t k = k0 + u * blockDim.x;
            mode[u] = 0;
            if (k < k_end && k < carry_units) {
                const uint32_t r = k / upr;
                colf[u] = 16u * (k - r * upr);
                L[u] = row_len(a, r);
                mrow[u] = a.msg_in + (uint64_t)r * a.Q;
                if (colf[u] < 4 * L[u]) {
                    i0[u] = quarter(colf[u], L[u]);
                    if (colf[u] + 15 < 4 * L[u] && quarter(colf[u] + 15, L[u]) == i0[u]) {
                        mode[u] = 1;
                        load16(mrow[u] + (colf[u] - i0[u] * L[u]), m[u]);
                    } else {
                        mode[u] = 2;
                    }
                }
            }
        }
        if constexpr (INPLACE) {
#pragma unroll
            for (int u = 0; u < UT; ++u) {
                if (mode[u]) {
                    const uint32_t k = k0 + u * blockDim.x;
#pragma unroll
                    for (int q = 0; q < CH; ++q)
                        c[u][q] = __ldcs(src + (uint64_t)k * CH + q);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < UT; ++u) {
            const uint32_t k = k0 + u * blockDim.x;
            if (k >= k_end || (INPLACE && !mode[u]))
                continue;
            uint4 o[CH];
#pragma unroll
            for (int q = 0; q < CH; ++q)
                o[q] = c[u][q];
            if (mode[u] == 1) {
                uint32_t P[4];
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    P[q] = (m[u][q] >> (2 * i0[u])) & 0x03030303u;
                if (CH == 1) {
                    o[0].x = (o[0].x & 0xFCFCFCFCu) | P[0];
                    o[0].y = (o[0].y & 0xFCFCFCFCu) | P[1];
                    o[0].z = (o[0].z & 0xFCFCFCFCu) | P[2];
                    o[0].w = (o[0].w & 0xFCFCFCFCu) | P[3];
                } else {
                    put_unit<CH, PLANE, 0>(o, P);
                }
            } else if (mode[u] == 2) {
                slow_unit<CH, PLANE, 0>(o, colf[u], L[u], mrow[u]);
            }
            if (STATS && mode[u]) {
                uint32_t n = 0, sq = 0; // at most 16 pairs changed, 9 each
#pragma unroll
                for (int q = 0; q < CH; ++q)
                    pair_stats(o[q], c[u][q], n, sq);
                changed += n;
                sse += sq;
            }
#pragma unroll
            for (int q = 0; q < CH; ++q)
                __stcs(dst + (uint64_t)k * CH + q, o[q]);
        }
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
                if (CH == 1) {
                    P[0] = c[i][0].x & 0x03030303u;
                    P[1] = c[i][0].y & 0x03030303u;
                    P[2] = c[i][0].z & 0x03030303u;
                    P[3] = c[i][0].w & 0x03030303u;
                } else {
                    get_unit<CH, PLANE, 0>(c[i], P);
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
