// paper2.cu -- Sections VI and VII as printed: two bits per cover byte in one
// colour plane, the message divided greedily among image rows.
//
// Row r of plane `plane` is A_r[x] = cover[(r*W + x)*channels + plane].  With
// Q = floor(W/4) (Section VI step 5: 4*|B| <= |A|), rows take Q message bytes
// each until fewer than Q remain (Section VII step 4): the first R - 1 rows
// take Q, row R - 1 takes L_last = N - (R-1)*Q, later rows none.  Block i of
// the paper's launch writes bit pair i of B[j] to A_r[L_r*i + j] (Section VI
// step 7); extraction ORs the pairs back (Section VII step 6).
//
// Kernels.  Rows are the unit of work, as in the paper; the per-byte path
// has no integer division.
//   p2_embed_units<CH,PLANE>  out of place, 16-byte aligned buffers, W a
//       multiple of 16, CH in {1,3,4}: one pass over the image in units of
//       16 pixels (CH 16-byte vectors), persistent grid.  Pixel t of a unit
//       keeps its plane byte at unit byte t*CH + PLANE, a compile-time
//       position.  A unit inside one quarter of a carrying row takes its 16
//       pairs from 16 consecutive message bytes with four 32-bit loads and a
//       SWAR shift-and-mask; units across a quarter boundary or the end of
//       the carrying columns go pixel by pixel.  Traffic 2C + N.
//   p2_embed_rows  in place (and the fallback after a copy): thread j of row
//       r reads B[r*Q + j] once and rewrites its four plane bytes, four
//       message bytes per thread in flight.
//   p2_extract_units<CH,PLANE>  runs of 16 message bytes: the thread reads
//       the four units at columns i*L + j0 (i = 0..3) and ORs their pairs;
//       runs that are not whole aligned units go byte by byte.
//   p2_extract_rows  any channel count: thread j of row r gathers its four
//       pairs into B[r*Q + j].
#include "internal.cuh"

namespace stego {
namespace {

struct P2Args {
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
    stego_result *res;
};

__device__ __forceinline__ uint32_t row_len(const P2Args &a, uint32_t r)
{
    return r + 1 < a.R ? a.Q : (r + 1 == a.R ? a.L_last : 0u);
}

__device__ __forceinline__ void write_res(const P2Args &a, bool stats)
{
    if (a.res && blockIdx.x == 0 && threadIdx.x == 0) {
        a.res->msg_bytes = a.N;
        a.res->status = STEGO_OK;
        a.res->reserved = 0;
        if (!stats) {
            a.res->changed = 0;
            a.res->sse = 0;
        }
    }
}

// Quarter of a carrying column (block i of the paper): 0..3.
__device__ __forceinline__ uint32_t quarter(uint32_t col, uint32_t L)
{
    return (col >= L) + (col >= 2 * L) + (col >= 3 * L);
}

// ---------------------------------------------------------------------------
// One-pass kernels over units of 16 consecutive pixels of a row (CH 16-byte
// vectors).  Pixel t of a unit has its plane byte at unit byte t*CH + PLANE,
// a compile-time position once CH and PLANE are template parameters.
// ---------------------------------------------------------------------------

// Byte b (compile-time) of a unit of CH vectors, as a reference to its word.
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
// low two bits of some bytes.
__device__ __forceinline__ void pair_stats(const uint4 &o, const uint4 &c,
                                           unsigned long long &changed, unsigned long long &sse)
{
    const uint32_t ow[4] = {o.x, o.y, o.z, o.w}, cw[4] = {c.x, c.y, c.z, c.w};
    uint32_t n = 0, s = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint32_t x = ow[q] ^ cw[q];
        n += __popc((x | (x >> 1)) & 0x01010101u);
        const uint32_t d = __vabsdiffu4(ow[q] & 0x03030303u, cw[q] & 0x03030303u);
        s = __dp4a(d, d, s);
    }
    changed += n;
    sse += s;
}

// Out of place, one pass: every unit of the image is loaded and stored; the
// plane bytes of carrying units get their pairs on the way.  Each thread
// issues the cover loads of its UT units, then their message loads, before
// any arithmetic, so both latencies overlap.
template <int CH, int PLANE, bool STATS>
__global__ void __launch_bounds__(256, 3) p2_embed_units(P2Args a)
{
    constexpr int UT = 2; // units per thread in flight
    unsigned long long changed = 0, sse = 0;
    write_res(a, STATS);
    const uint32_t upr = a.W / 16; // units per row
    const uint32_t nunits = upr * a.H;        // < 2^32 (checked by the launcher)
    const uint32_t carry_units = upr * a.R;
    const uint4 *__restrict__ src = reinterpret_cast<const uint4 *>(a.src);
    uint4 *dst = reinterpret_cast<uint4 *>(a.dst);
    const uint32_t stride = gridDim.x * blockDim.x * UT;
    for (uint32_t k0 = blockIdx.x * blockDim.x * UT + threadIdx.x; k0 < nunits; k0 += stride) {
        uint4 c[UT][CH];
#pragma unroll
        for (int u = 0; u < UT; ++u) {
            const uint32_t k = k0 + u * blockDim.x;
            if (k < nunits) {
#pragma unroll
                for (int q = 0; q < CH; ++q)
                    c[u][q] = __ldcs(src + (uint64_t)k * CH + q);
            }
        }
        // 0: copy only, 1: one quarter (SWAR), 2: per pixel
        int mode[UT];
        uint32_t colf[UT], L[UT], i0[UT], m[UT][4];
        const uint8_t *mrow[UT];
#pragma unroll
        for (int u = 0; u < UT; ++u) {
            const uint32_t k = k0 + u * blockDim.x;
            mode[u] = 0;
            if (k < carry_units) {
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
#pragma unroll
        for (int u = 0; u < UT; ++u) {
            const uint32_t k = k0 + u * blockDim.x;
            if (k >= nunits)
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
#pragma unroll
                for (int q = 0; q < CH; ++q)
                    pair_stats(o[q], c[u][q], changed, sse);
            }
#pragma unroll
            for (int q = 0; q < CH; ++q)
                __stcs(dst + (uint64_t)k * CH + q, o[q]);
        }
    }
    if (STATS)
        block_add2(changed, sse, reinterpret_cast<unsigned long long *>(&a.res->changed));
}

// Extraction over runs of 16 message bytes: the thread owning B[j0..j0+15]
// of row r reads the four units (quarters i = 0..3) at columns i*L + j0 and
// ORs their pairs into the bytes.  Runs that are not whole aligned units
// (the last row, or quarters not on 16-byte boundaries) take the per-byte
// path.
template <int CH, int PLANE>
__global__ void __launch_bounds__(512) p2_extract_units(P2Args a)
{
    if (a.res && blockIdx.x == 0 && threadIdx.x == 0) {
        a.res->changed = 0;
        a.res->sse = 0;
        a.res->msg_bytes = a.N;
        a.res->status = STEGO_OK;
        a.res->reserved = 0;
    }
    const uint32_t rpr = (a.Q + 15) / 16; // runs per full row
    const uint64_t nruns = (uint64_t)rpr * a.R;
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nruns;
         k += (uint64_t)gridDim.x * blockDim.x) {
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
                    const uint32_t *w = reinterpret_cast<const uint32_t *>(&c[i][0]);
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        P[q] = w[q] & 0x03030303u;
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

template <bool STATS>
__global__ void __launch_bounds__(512, 2) p2_embed_rows(P2Args a)
{
    unsigned long long changed = 0, sse = 0;
    write_res(a, STATS);
    for (uint32_t r = blockIdx.x; r < a.R; r += gridDim.x) {
        const uint32_t L = row_len(a, r);
        const uint8_t *mrow = a.msg_in + (uint64_t)r * a.Q;
        const uint64_t prow = (uint64_t)r * a.W;
        constexpr int U = 4; // message bytes per thread in flight
        for (uint32_t j0 = threadIdx.x; j0 < L; j0 += blockDim.x * U) {
            // byte of pair i of B[j]: base(j) + i*qstride
            const uint64_t qstride = (uint64_t)L * a.channels;
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
    if (STATS)
        block_add2(changed, sse, reinterpret_cast<unsigned long long *>(&a.res->changed));
}

__global__ void __launch_bounds__(512) p2_extract_rows(P2Args a)
{
    if (a.res && blockIdx.x == 0 && threadIdx.x == 0) {
        a.res->changed = 0;
        a.res->sse = 0;
        a.res->msg_bytes = a.N;
        a.res->status = STEGO_OK;
        a.res->reserved = 0;
    }
    for (uint32_t r = blockIdx.x; r < a.R; r += gridDim.x) {
        const uint32_t L = row_len(a, r);
        uint8_t *mrow = a.msg_out + (uint64_t)r * a.Q;
        const uint64_t prow = (uint64_t)r * a.W;
        constexpr int U = 4; // message bytes per thread in flight
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

P2Args make_args(const uint8_t *src, uint8_t *dst, const stego_geom &g, const uint8_t *msg_in,
                 uint8_t *msg_out, uint64_t N, stego_result *res)
{
    P2Args a;
    a.src = src;
    a.dst = dst;
    a.msg_in = msg_in;
    a.msg_out = msg_out;
    a.N = N;
    a.W = g.width;
    a.H = g.height;
    a.channels = g.channels;
    a.plane = g.plane;
    a.Q = g.width / 4u;
    a.R = a.Q ? (uint32_t)((N + a.Q - 1) / a.Q) : 0u;
    a.L_last = a.R ? (uint32_t)(N - (uint64_t)(a.R - 1) * a.Q) : 0u;
    a.pad = 0;
    a.res = res;
    return a;
}

int row_grid(const void *k, const Shape &sh, uint32_t rows)
{
    return persistent_grid(k, sh.threads, 0, sh.ctas_per_sm, rows ? rows : 1, 1);
}

} // namespace

bool p2_fused_ok(const uint8_t *cover, const uint8_t *stego, const stego_geom &g)
{
    const uint32_t ch = g.channels;
    // units of 16 pixels are counted in 32 bits (plus a stride of headroom)
    return cover != stego && ((((uintptr_t)cover | (uintptr_t)stego) & 15u) == 0) &&
           (ch == 1 || ch == 3 || ch == 4) && g.width % 16u == 0 &&
           (uint64_t)g.width / 16u * g.height < (1ull << 31);
}

namespace {

template <bool STATS>
const void *units_kernel(uint32_t ch, uint32_t plane)
{
    if (ch == 1)
        return (const void *)p2_embed_units<1, 0, STATS>;
    if (ch == 3) {
        switch (plane) {
        case 0: return (const void *)p2_embed_units<3, 0, STATS>;
        case 1: return (const void *)p2_embed_units<3, 1, STATS>;
        default: return (const void *)p2_embed_units<3, 2, STATS>;
        }
    }
    switch (plane) {
    case 0: return (const void *)p2_embed_units<4, 0, STATS>;
    case 1: return (const void *)p2_embed_units<4, 1, STATS>;
    case 2: return (const void *)p2_embed_units<4, 2, STATS>;
    default: return (const void *)p2_embed_units<4, 3, STATS>;
    }
}

const void *extract_units_kernel(uint32_t ch, uint32_t plane)
{
    if (ch == 1)
        return (const void *)p2_extract_units<1, 0>;
    if (ch == 3) {
        switch (plane) {
        case 0: return (const void *)p2_extract_units<3, 0>;
        case 1: return (const void *)p2_extract_units<3, 1>;
        default: return (const void *)p2_extract_units<3, 2>;
        }
    }
    switch (plane) {
    case 0: return (const void *)p2_extract_units<4, 0>;
    case 1: return (const void *)p2_extract_units<4, 1>;
    case 2: return (const void *)p2_extract_units<4, 2>;
    default: return (const void *)p2_extract_units<4, 3>;
    }
}

} // namespace

cudaError_t p2_embed_fused(const uint8_t *cover, uint8_t *stego, const stego_geom &g,
                           const uint8_t *msg, uint64_t N, bool stats, stego_result *res,
                           const Shape &sh, cudaStream_t s)
{
    P2Args a = make_args(cover, stego, g, msg, nullptr, N, res);
    const void *k = stats ? units_kernel<true>(g.channels, g.plane)
                          : units_kernel<false>(g.channels, g.plane);
    const uint64_t nunits = (uint64_t)(g.width / 16u) * g.height;
    const int threads = 256; // the kernel's register bound assumes 256
    const int grid = persistent_grid(k, threads, 0, sh.ctas_per_sm, nunits ? nunits : 1,
                                     (uint64_t)threads * 2);
    void *args[] = {&a};
    return cudaLaunchKernel(k, dim3(grid), dim3(threads), args, 0, s);
}

cudaError_t p2_embed(const uint8_t *cover, uint8_t *stego, const stego_geom &g,
                     const uint8_t *msg, uint64_t N, bool stats, stego_result *res,
                     const Shape &sh, cudaStream_t s)
{
    P2Args a = make_args(cover, stego, g, msg, nullptr, N, res);
    const void *k = stats ? (const void *)p2_embed_rows<true> : (const void *)p2_embed_rows<false>;
    const int grid = row_grid(k, sh, a.R);
    void *args[] = {&a};
    return cudaLaunchKernel(k, dim3(grid), dim3(sh.threads), args, 0, s);
}

cudaError_t p2_extract(const uint8_t *st, const stego_geom &g, uint8_t *msg, uint64_t N,
                       stego_result *res, const Shape &sh, cudaStream_t s)
{
    P2Args a = make_args(st, nullptr, g, nullptr, msg, N, res);
    const uint32_t ch = g.channels;
    if (ch == 1 || ch == 3 || ch == 4) {
        const void *k = extract_units_kernel(ch, g.plane);
        const uint64_t runs = (uint64_t)((a.Q + 15) / 16) * a.R;
        const int grid = persistent_grid(k, sh.threads, 0, sh.ctas_per_sm, runs ? runs : 1,
                                         (uint64_t)sh.threads);
        void *args[] = {&a};
        return cudaLaunchKernel(k, dim3(grid), dim3(sh.threads), args, 0, s);
    }
    const void *k = (const void *)p2_extract_rows;
    const int grid = row_grid(k, sh, a.R);
    void *args[] = {&a};
    return cudaLaunchKernel(k, dim3(grid), dim3(sh.threads), args, 0, s);
}

} // namespace stego
