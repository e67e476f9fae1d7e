// batched.cu -- many covers or video frames of uneven sizes in one persistent
// launch.  The paper runs its routine once per image row and per frame
// (Section VI, last paragraph; image/video frames, Section III) with a
// device allocation, two copies and a launch each time; here every cover of
// a batch is cut into fixed-size tiles that one persistent grid claims from
// a work counter.
//
// Per call, stream-ordered launches (all capturable in a CUDA graph):
//   1. prep      one thread per descriptor: validate it, (extract) read its
//                32-bit header, write its result and its tile count;
//   2. scan      one CTA: exclusive scan of the tile counts into tile
//                offsets, total, work counter reset;
//   3. persist   SMs x occupancy CTAs: claim `chunk` consecutive tiles at a
//                time with one atomicAdd (the next claim is issued while the
//                current chunk is processed), find the owning descriptor by
//                binary search over the offsets once per chunk, and run the
//                same per-vector code as the single-cover kernels on each
//                tile; one persistent kernel per tile space (one-bit stream
//                on 16-byte aligned buffers, one-bit stream on misaligned
//                buffers, paper layout), each exiting at once when its space
//                is empty.
// Workspace (caller-owned scratch, 16-byte aligned):
//   [0, 64)                 head: tile totals and work counters
//   [64, 64 + 24(n+1))      tile offsets of the three spaces (counts before
//                           the scan)
//   [info_off, +64n)        per-descriptor derived sizes, geometry and mode
// Both layouts batch: the one-bit stream in tiles of cover bytes; the
// paper's layout (Sections VI/VII) in tiles of whole rows (copy, barrier,
// scatter out of place; scatter in place) and, for extraction, of 16-byte
// message runs (1, 3 or 4 channels) or rows, with the routines the
// single-image kernels use.  The paper layout has its own persistent
// kernels (own tile offsets and counter), so its register needs do not
// touch the stream kernels'.
#include <cstring>
#include <mutex>

#include "p2_device.cuh"
#include "s1_device.cuh"

namespace stego {
namespace {

struct WsHead {
    unsigned long long total;     // one-bit stream tiles, aligned buffers
    unsigned long long counter;
    unsigned long long total_p;   // paper-layout tiles
    unsigned long long counter_p;
    unsigned long long total_m;   // one-bit stream tiles, misaligned buffers
    unsigned long long counter_m;
    unsigned long long pad[2];
};

struct DescInfo {
    uint64_t n_bytes; // stream embed: bytes written; stream extract: 8*len
    uint64_t t_bytes; // stream embed: carrying bytes
    uint64_t len;     // stream embed: stream bytes; extract / paper: message bytes
    uint32_t nbits;   // header value
    uint32_t bits;    // kHeader | kVec | kMsgEven | kFunnel
    uint32_t W, H;    // paper layout geometry; misaligned stream: head bytes,
                      // funnel byte selector
    uint32_t channels, plane; // misaligned stream embed: channels = Q (funnel word offset)
    uint32_t mode;     // paper layout: one of the kP2* work kinds
    uint32_t per_tile; // paper layout: units, rows or runs per tile
    uint32_t pad[2];
};
static_assert(sizeof(DescInfo) == 64, "DescInfo is 64 bytes");

constexpr uint32_t kHeader = 1u, kVec = 2u, kMsgEven = 4u;
// misaligned stream embed: cover and stego at different addresses mod 16
// (stego vectors joined from cover vector pairs); otherwise the same
// misalignment (vectors after a scalar head)
constexpr uint32_t kFunnel = 8u;
// paper-layout work kinds (0 = the one-bit stream layout)
constexpr uint32_t kP2Units = 1u, kP2RowsCopy = 2u, kP2Rows = 3u, kP2Runs = 4u, kP2RowsX = 5u,
                   kP2UnitsInPlace = 6u;
// Threads of the paper-layout persistent kernels' CTAs.  Unit and run tiles
// hold a whole number of CTA rounds (tile_bytes rounded down), so that no
// round runs with idle threads in the middle of a cover.
constexpr uint32_t kP2Threads = 256u;
__device__ __forceinline__ uint64_t whole_rounds(uint64_t per)
{
    return per >= kP2Threads ? per / kP2Threads * kP2Threads : per;
}
constexpr uint32_t kChunk = 4u; // tiles per claim

// Workspace: head (64 B), aligned-stream, paper and misaligned-stream tile
// offsets (n+1 each), per-descriptor info (64 B each, 16-byte aligned).
constexpr uint64_t startp_off(uint32_t n) { return 64ull + 8ull * ((uint64_t)n + 1); }
constexpr uint64_t startm_off(uint32_t n) { return 64ull + 16ull * ((uint64_t)n + 1); }
constexpr uint64_t info_off(uint32_t n)
{
    return (64ull + 24ull * ((uint64_t)n + 1) + 15ull) & ~15ull;
}

struct WsView {
    WsHead *head;
    unsigned long long *start;   // stream-layout tile offsets, aligned buffers
    unsigned long long *start_p; // paper-layout tile offsets
    unsigned long long *start_m; // stream-layout tile offsets, misaligned buffers
    DescInfo *info;
};

WsView ws_view(void *ws, uint32_t n)
{
    WsView v;
    v.head = reinterpret_cast<WsHead *>(ws);
    v.start = reinterpret_cast<unsigned long long *>((char *)ws + 64);
    v.start_p = reinterpret_cast<unsigned long long *>((char *)ws + startp_off(n));
    v.start_m = reinterpret_cast<unsigned long long *>((char *)ws + startm_off(n));
    v.info = reinterpret_cast<DescInfo *>((char *)ws + info_off(n));
    return v;
}

__device__ __forceinline__ bool d_overlap(const void *p, uint64_t np, const void *q, uint64_t nq)
{
    if (np == 0 || nq == 0 || p == nullptr || q == nullptr)
        return false;
    const uintptr_t a = (uintptr_t)p, b = (uintptr_t)q;
    return a < b + nq && b < a + np;
}

__device__ __forceinline__ bool d_aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// ---------------------------------------------------------------------------
// 1. prep
// ---------------------------------------------------------------------------

__device__ __forceinline__ void clear_info(DescInfo &inf)
{
    inf.n_bytes = inf.t_bytes = inf.len = 0;
    inf.nbits = inf.bits = 0;
    inf.W = inf.H = inf.channels = inf.plane = 0;
    inf.mode = inf.per_tile = 0;
    inf.pad[0] = inf.pad[1] = 0;
}

// Paper-layout geometry of a descriptor: channels > 0, plane < channels and
// width * height * channels == cover_bytes (Section VI step 2).
__device__ __forceinline__ bool paper_geom_ok(const stego_desc &D)
{
    const stego_geom &g = D.geom;
    return g.channels > 0 && g.plane < g.channels &&
           (uint64_t)g.width * g.height * g.channels == D.cover_bytes;
}

__device__ __forceinline__ void paper_info(const stego_desc &D, DescInfo &inf, uint64_t N)
{
    inf.len = N;
    inf.W = D.geom.width;
    inf.H = D.geom.height;
    inf.channels = D.geom.channels;
    inf.plane = D.geom.plane;
}

// Whole rows per tile for the row-based work kinds (at least one).
__device__ __forceinline__ uint64_t rows_for(const stego_desc &D, uint32_t tile_bytes)
{
    const uint64_t rb = (uint64_t)D.geom.width * D.geom.channels;
    const uint64_t r = rb ? tile_bytes / rb : 1u;
    return r ? r : 1u;
}

__global__ void prep_embed(const stego_desc *descs, uint32_t n, stego_result *results, WsView ws,
                           uint32_t tile_bytes)
{
    grid_dependency_wait(); // launched dependent: nothing is touched before
    allow_dependents();
    for (uint32_t d = blockIdx.x * blockDim.x + threadIdx.x; d < n; d += gridDim.x * blockDim.x) {
        const stego_desc D = descs[d];
        const uint32_t layout = D.flags & STEGO_LAYOUT_MASK;
        const bool header = (D.flags & STEGO_HEADER_BE32) != 0;
        const bool inplace = D.stego == D.cover;
        int st = STEGO_OK;
        if (D.flags & ~(STEGO_LAYOUT_MASK | STEGO_HEADER_BE32 | STEGO_FUSE_STATS))
            st = STEGO_E_INVAL;
        else if (layout != STEGO_LAYOUT_STREAM1 && layout != STEGO_LAYOUT_PAPER2)
            st = STEGO_E_INVAL;
        else if (D.cover_bytes > 0 && (!D.cover || !D.stego))
            st = STEGO_E_INVAL;
        else if (D.msg_bytes > 0 && !D.msg)
            st = STEGO_E_INVAL;
        else if (!inplace && d_overlap(D.cover, D.cover_bytes, D.stego, D.cover_bytes))
            st = STEGO_E_INVAL;
        else if (d_overlap(D.msg, D.msg_bytes, D.stego, D.cover_bytes))
            st = STEGO_E_INVAL;
        else if (layout == STEGO_LAYOUT_PAPER2) {
            if (header || !paper_geom_ok(D))
                st = STEGO_E_INVAL;
            else if (D.msg_bytes > (uint64_t)(D.geom.width / 4u) * D.geom.height)
                st = STEGO_E_CAPACITY;
        } else {
            uint64_t cap = D.cover_bytes / 8u;
            if (header) {
                cap = cap >= 4u ? cap - 4u : 0u;
                if (cap > 0x1FFFFFFFull)
                    cap = 0x1FFFFFFFull;
            }
            if (D.msg_bytes > cap || (header && D.cover_bytes < 32))
                st = STEGO_E_CAPACITY;
        }
        DescInfo inf;
        clear_info(inf);
        unsigned long long tiles = 0;
        if (st == STEGO_OK && layout == STEGO_LAYOUT_PAPER2) {
            paper_info(D, inf, D.msg_bytes);
            const uint32_t ch = D.geom.channels;
            const uint64_t rows_per_tile = rows_for(D, tile_bytes);
            const p2::View v = p2::make_view(nullptr, nullptr, D.geom.width, D.geom.height, ch,
                                             D.geom.plane, nullptr, nullptr, D.msg_bytes);
            if (!inplace && d_aligned16(D.cover) && d_aligned16(D.stego) &&
                (ch == 3 || ch == 1) && D.geom.width % 16u == 0 &&
                (uint64_t)D.geom.width / 16u * D.geom.height < (1ull << 31)) {
                // one-pass units: grayscale, or RGB with any plane
                const uint64_t units = (uint64_t)(D.geom.width / 16u) * D.geom.height;
                const uint64_t per =
                    whole_rounds(tile_bytes / (16u * ch) ? tile_bytes / (16u * ch) : 1u);
                inf.mode = kP2Units;
                inf.per_tile = (uint32_t)per;
                tiles = (units + per - 1) / per;
            } else if (inplace && d_aligned16(D.cover) && (ch == 3 || ch == 1) &&
                       D.geom.width % 16u == 0 &&
                       (uint64_t)D.geom.width / 16u * D.geom.height < (1ull << 31)) {
                // in place: the units of the carrying rows, written back whole
                const uint64_t units = (uint64_t)(D.geom.width / 16u) * v.R;
                const uint64_t per =
                    whole_rounds(tile_bytes / (16u * ch) ? tile_bytes / (16u * ch) : 1u);
                inf.mode = kP2UnitsInPlace;
                inf.per_tile = (uint32_t)per;
                tiles = (units + per - 1) / per;
            } else if (!inplace) {
                inf.mode = kP2RowsCopy;
                inf.per_tile = (uint32_t)rows_per_tile;
                tiles = (D.geom.height + rows_per_tile - 1) / rows_per_tile;
            } else {
                inf.mode = kP2Rows;
                inf.per_tile = (uint32_t)rows_per_tile;
                tiles = (v.R + rows_per_tile - 1) / rows_per_tile;
            }
        } else if (st == STEGO_OK) {
            inf.len = D.msg_bytes + (header ? 4u : 0u);
            inf.t_bytes = 8u * inf.len;
            inf.n_bytes = inplace ? inf.t_bytes : D.cover_bytes;
            inf.nbits = (uint32_t)(8u * D.msg_bytes);
            inf.bits = (header ? kHeader : 0u) |
                       ((d_aligned16(D.cover) && d_aligned16(D.stego)) ? kVec : 0u) |
                       ((((uintptr_t)D.msg & 1u) == 0) ? kMsgEven : 0u);
            tiles = (inf.n_bytes + tile_bytes - 1) / tile_bytes;
            if (!(inf.bits & kVec)) {
                // misaligned: aligned vectors after h head bytes, in tiles
                // of tile_bytes/16 vectors, when at least one vector fits
                const uint32_t hc = (uint32_t)((16u - ((uintptr_t)D.cover & 15u)) & 15u);
                const uint32_t hs = (uint32_t)((16u - ((uintptr_t)D.stego & 15u)) & 15u);
                const bool same = (((uintptr_t)D.cover ^ (uintptr_t)D.stego) & 15u) == 0;
                const uint32_t h = same ? hc : hs;
                if ((same || !inplace) && inf.n_bytes >= (uint64_t)h + 16u) {
                    const uint64_t nvb = (inf.n_bytes - h) >> 4;
                    const uint64_t tv = tile_bytes / 16u;
                    inf.W = h;
                    if (!same) {
                        const uint32_t dd = (uint32_t)(((uintptr_t)D.cover + hs) & 15u);
                        const uint32_t b = dd & 3u;
                        inf.bits |= kFunnel;
                        inf.H = b | ((b + 1) << 4) | ((b + 2) << 8) | ((b + 3) << 12);
                        inf.channels = dd >> 2;
                    }
                    inf.per_tile = (uint32_t)tv;
                    inf.mode = 0;
                    ws.info[d] = inf;
                    ws.start[d] = 0ull;
                    ws.start_p[d] = 0ull;
                    ws.start_m[d] = (nvb + tv - 1) / tv;
                    stego_result r;
                    r.changed = 0;
                    r.sse = 0;
                    r.msg_bytes = D.msg_bytes;
                    r.status = STEGO_OK;
                    r.reserved = 0;
                    results[d] = r;
                    continue;
                }
            }
        }
        ws.info[d] = inf;
        ws.start[d] = inf.mode ? 0ull : tiles;
        ws.start_p[d] = inf.mode ? tiles : 0ull;
        ws.start_m[d] = 0ull;
        stego_result r;
        r.changed = 0;
        r.sse = 0;
        r.msg_bytes = st == STEGO_OK ? D.msg_bytes : 0u;
        r.status = st;
        r.reserved = 0;
        results[d] = r;
    }
}

__global__ void prep_extract(const stego_desc *descs, uint32_t n, stego_result *results,
                             WsView ws, uint32_t tile_bytes)
{
    grid_dependency_wait(); // launched dependent: nothing is touched before
    allow_dependents();
    for (uint32_t d = blockIdx.x * blockDim.x + threadIdx.x; d < n; d += gridDim.x * blockDim.x) {
        const stego_desc D = descs[d];
        const uint32_t layout = D.flags & STEGO_LAYOUT_MASK;
        const bool header = (D.flags & STEGO_HEADER_BE32) != 0;
        int st = STEGO_OK;
        uint64_t len = 0;
        uint32_t nbits = 0;
        if (D.flags & ~(STEGO_LAYOUT_MASK | STEGO_HEADER_BE32 | STEGO_FUSE_STATS))
            st = STEGO_E_INVAL;
        else if (layout != STEGO_LAYOUT_STREAM1 && layout != STEGO_LAYOUT_PAPER2)
            st = STEGO_E_INVAL;
        else if (layout == STEGO_LAYOUT_PAPER2 && (header || !paper_geom_ok(D)))
            st = STEGO_E_INVAL;
        else if (D.cover_bytes > 0 && !D.cover)
            st = STEGO_E_INVAL;
        else if (D.msg_bytes > 0 && !D.msg)
            st = STEGO_E_INVAL;
        else if (d_overlap(D.msg, D.msg_bytes, D.cover, D.cover_bytes))
            st = STEGO_E_INVAL;
        else if (layout == STEGO_LAYOUT_PAPER2) {
            len = D.msg_len;
            if (len > (uint64_t)(D.geom.width / 4u) * D.geom.height)
                st = STEGO_E_CAPACITY;
            else if (len > D.msg_bytes)
                st = STEGO_E_MSG_TOO_SMALL;
        } else if (header) {
            if (D.cover_bytes < 32) {
                st = STEGO_E_BAD_HEADER;
            } else {
                for (int k = 0; k < 32; ++k)
                    nbits |= (uint32_t)(D.cover[k] & 1u) << (31 - k);
                st = s1::header_status(D.cover_bytes, D.msg_bytes, nbits);
                len = nbits >> 3;
            }
        } else {
            len = D.msg_len;
            if (len > D.cover_bytes / 8u)
                st = STEGO_E_CAPACITY;
            else if (len > D.msg_bytes)
                st = STEGO_E_MSG_TOO_SMALL;
        }
        if (st != STEGO_OK)
            len = 0;
        DescInfo inf;
        clear_info(inf);
        unsigned long long tiles = 0;
        if (layout == STEGO_LAYOUT_PAPER2 && st == STEGO_OK) {
            paper_info(D, inf, len);
            const p2::View v = p2::make_view(nullptr, nullptr, D.geom.width, D.geom.height,
                                             D.geom.channels, D.geom.plane, nullptr, nullptr, len);
            if (p2::unit_channels(D.geom.channels)) {
                const uint64_t runs = (uint64_t)((v.Q + 15) / 16) * v.R;
                const uint64_t per = whole_rounds(tile_bytes / (64u * D.geom.channels)
                                                      ? tile_bytes / (64u * D.geom.channels)
                                                      : 1u);
                inf.mode = kP2Runs;
                inf.per_tile = (uint32_t)per;
                tiles = (runs + per - 1) / per;
            } else {
                const uint64_t per = rows_for(D, tile_bytes);
                inf.mode = kP2RowsX;
                inf.per_tile = (uint32_t)per;
                tiles = (v.R + per - 1) / per;
            }
        } else {
            inf.len = len;
            inf.n_bytes = 8u * len;
            inf.nbits = nbits;
            const uint8_t *carrying = D.cover + (header ? 32u : 0u);
            inf.bits = (header ? kHeader : 0u) | (d_aligned16(carrying) ? kVec : 0u) |
                       ((((uintptr_t)D.msg & 1u) == 0) ? kMsgEven : 0u);
            tiles = (inf.n_bytes + tile_bytes - 1) / tile_bytes;
            if (!(inf.bits & kVec) && len >= 2) {
                // misaligned carrying bytes: message byte pairs from aligned
                // vector pairs, in tiles of tile_bytes/16 pairs
                const uint64_t tv = tile_bytes / 16u;
                inf.per_tile = (uint32_t)tv;
                ws.info[d] = inf;
                ws.start[d] = 0ull;
                ws.start_p[d] = 0ull;
                ws.start_m[d] = ((len >> 1) + tv - 1) / tv;
                stego_result r;
                r.changed = 0;
                r.sse = 0;
                r.msg_bytes = len;
                r.status = st;
                r.reserved = 0;
                results[d] = r;
                continue;
            }
        }
        ws.info[d] = inf;
        ws.start[d] = inf.mode ? 0ull : tiles;
        ws.start_p[d] = inf.mode ? tiles : 0ull;
        ws.start_m[d] = 0ull;
        stego_result r;
        r.changed = 0;
        r.sse = 0;
        r.msg_bytes = len;
        r.status = st;
        r.reserved = 0;
        results[d] = r;
    }
}

// ---------------------------------------------------------------------------
// 2. scan (one CTA of kScanThreads)
// ---------------------------------------------------------------------------

constexpr int kScanThreads = 1024;

// Exclusive scan of counts[0..n) in place, counts[n] = total; the calling
// CTA's kScanThreads threads together.
__device__ __forceinline__ unsigned long long scan_one(unsigned long long *counts, uint32_t n,
                                                      unsigned long long *part)
{
    const uint32_t t = threadIdx.x, T = blockDim.x;
    const uint64_t seg = ((uint64_t)n + T - 1) / T;
    const uint64_t b = (uint64_t)t * seg;
    const uint64_t e = b + seg < n ? b + seg : n;
    unsigned long long sum = 0;
    for (uint64_t i = b; i < e; ++i)
        sum += counts[i];
    part[t] = sum;
    __syncthreads();
    for (uint32_t off = 1; off < T; off <<= 1) {
        const unsigned long long v = t >= off ? part[t - off] : 0ull;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    unsigned long long run = part[t] - sum;
    for (uint64_t i = b; i < e; ++i) {
        const unsigned long long c = counts[i];
        counts[i] = run;
        run += c;
    }
    const unsigned long long total = part[T - 1];
    if (t == T - 1)
        counts[n] = total;
    __syncthreads(); // part[] is reused by the next scan
    return total;
}

__global__ void __launch_bounds__(kScanThreads) scan_tiles(WsView ws, uint32_t n)
{
    grid_dependency_wait(); // launched dependent: nothing is touched before
    allow_dependents();
    __shared__ unsigned long long part[kScanThreads];
    const unsigned long long ts = scan_one(ws.start, n, part);
    const unsigned long long tp = scan_one(ws.start_p, n, part);
    const unsigned long long tm = scan_one(ws.start_m, n, part);
    if (threadIdx.x == 0) {
        ws.head->total = ts;
        ws.head->counter = 0;
        ws.head->total_p = tp;
        ws.head->counter_p = 0;
        ws.head->total_m = tm;
        ws.head->counter_m = 0;
    }
}

// ---------------------------------------------------------------------------
// 3. persistent kernels
// ---------------------------------------------------------------------------

// Largest d < n with start[d] <= t (start[0] = 0 <= t < start[n]).
__device__ __forceinline__ uint32_t owner_of(const unsigned long long *start, uint32_t n,
                                             unsigned long long t)
{
    uint32_t lo = 0, hi = n;
    while (hi - lo > 1) {
        const uint32_t mid = lo + ((hi - lo) >> 1);
        if (start[mid] <= t)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

// Warp-level flush of per-thread statistics into one descriptor's result.
__device__ __forceinline__ void flush_stats(unsigned long long &changed, unsigned long long &sse,
                                            stego_result *res)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        changed += __shfl_down_sync(0xFFFFFFFFu, changed, o);
        sse += __shfl_down_sync(0xFFFFFFFFu, sse, o);
    }
    if ((threadIdx.x & 31u) == 0 && res) {
        if (changed)
            atomicAdd(reinterpret_cast<unsigned long long *>(&res->changed), changed);
        if (sse)
            atomicAdd(reinterpret_cast<unsigned long long *>(&res->sse), sse);
    }
    changed = 0;
    sse = 0;
}

// The claim loop shared by both directions: calls body(d, local_tile) for
// every tile this CTA claims, in order.
template <typename Body>
__device__ __forceinline__ void claim_loop(const unsigned long long *start,
                                           unsigned long long total,
                                           unsigned long long *counter, uint32_t n, Body &&body)
{
    __shared__ unsigned long long s_claim;
    if (threadIdx.x == 0)
        s_claim = atomicAdd(counter, (unsigned long long)kChunk);
    __syncthreads();
    for (;;) {
        const unsigned long long c0 = s_claim;
        __syncthreads(); // every thread has read the claim
        if (c0 >= total)
            break;
        if (threadIdx.x == 0) // next claim in flight while this chunk runs
            s_claim = atomicAdd(counter, (unsigned long long)kChunk);
        const unsigned long long c1 = c0 + kChunk < total ? c0 + kChunk : total;
        uint32_t d = owner_of(start, n, c0);
        for (unsigned long long t = c0; t < c1; ++t) {
            while (start[d + 1] <= t)
                ++d;
            body(d, t - start[d]);
        }
        __syncthreads(); // the next claim is visible
    }
}

struct TileStats {
    unsigned long long changed, sse;
};

// The units of one tile of an RGB cover carrying in plane PLANE.
template <int PLANE, bool STATS>
__device__ __noinline__ TileStats rgb_units_tile(const p2::View v, uint32_t k0, uint32_t k1)
{
    TileStats t{0ull, 0ull};
    p2::units_embed<3, PLANE, STATS, 1>(v, k0, k1, blockDim.x, t.changed, t.sse);
    return t;
}

// One tile of a paper-layout cover (the CTA's threads together).
template <bool STATS>
__device__ __forceinline__ void paper_embed_tile(const stego_desc &D, const DescInfo &inf,
                                                 unsigned long long lt,
                                                 unsigned long long &changed,
                                                 unsigned long long &sse)
{
    const p2::View v = p2::make_view(D.cover, D.stego, inf.W, inf.H, inf.channels, inf.plane,
                                     D.msg, nullptr, inf.len);
    const uint64_t b0 = lt * inf.per_tile, b1 = b0 + inf.per_tile;
    if (inf.mode == kP2Units || inf.mode == kP2UnitsInPlace) {
        // in place the same code runs over the carrying rows' units only:
        // each unit is read and written back by one thread, so src == dst is
        // safe, and the last row's units past its carrying columns are
        // rewritten unchanged (one instantiation keeps the registers down)
        const bool ip = inf.mode == kP2UnitsInPlace;
        const uint64_t units = (uint64_t)(inf.W / 16u) * (ip ? v.R : inf.H);
        const uint32_t k0 = (uint32_t)b0 + threadIdx.x;
        const uint32_t k1 = (uint32_t)(b1 < units ? b1 : units);
        // one unit per thread, loaded by the thread itself: under the
        // 80-register cap a form staged through shared memory spilled more
        // and ran slower (600 video frames: 1.53 against 1.26 ms), and so did
        // the cp.async pipeline of the single-cover kernel (1.34-1.83 ms)
        if (inf.channels == 1) {
            p2::units_embed<1, 0, STATS, 1>(v, k0, k1, blockDim.x, changed, sse);
        } else if (inf.plane == 0) {
            p2::units_embed<3, 0, STATS, 1>(v, k0, k1, blockDim.x, changed, sse);
        } else {
            // planes 1 and 2 of RGB in calls of their own, so that their
            // registers do not crowd the plane-0 path (once per tile)
            const TileStats t = inf.plane == 1 ? rgb_units_tile<1, STATS>(v, k0, k1)
                                               : rgb_units_tile<2, STATS>(v, k0, k1);
            changed += t.changed;
            sse += t.sse;
        }
        return;
    }
    const uint32_t r0 = (uint32_t)b0;
    const uint32_t r1 = (uint32_t)(b1 < inf.H ? b1 : inf.H);
    if (inf.mode == kP2RowsCopy) {
        p2::rows_copy(v, r0, r1);
        __syncthreads(); // the copy lands before the scatter overwrites plane bytes
    }
    p2::rows_embed<STATS>(v, r0, r1, 1, changed, sse);
}

__device__ __forceinline__ void paper_extract_tile(const stego_desc &D, const DescInfo &inf,
                                                   unsigned long long lt)
{
    const p2::View v = p2::make_view(D.cover, nullptr, inf.W, inf.H, inf.channels, inf.plane,
                                     nullptr, D.msg, inf.len);
    const uint64_t b0 = lt * inf.per_tile, b1 = b0 + inf.per_tile;
    if (inf.mode == kP2Runs) {
        const uint64_t runs = (uint64_t)((v.Q + 15) / 16) * v.R;
        p2::runs_extract_any(v, b0 + threadIdx.x, b1 < runs ? b1 : runs, blockDim.x);
    } else {
        p2::rows_extract(v, (uint32_t)b0, (uint32_t)(b1 < v.R ? b1 : v.R), 1);
    }
}

template <int V, bool STATS>
__global__ void __launch_bounds__(512) persist_embed(const stego_desc *descs, uint32_t n,
                                                     stego_result *results, WsView ws,
                                                     uint32_t tile_bytes)
{
    grid_dependency_wait(); // launched dependent: nothing is touched before
    allow_dependents();
    unsigned long long changed = 0, sse = 0;
    uint32_t stat_d = 0xFFFFFFFFu;
    claim_loop(ws.start, ws.head->total, &ws.head->counter, n,
               [&](uint32_t d, unsigned long long lt) {
        if (STATS && d != stat_d) {
            flush_stats(changed, sse, stat_d < n ? results + stat_d : nullptr);
            stat_d = d;
        }
        const stego_desc &D = descs[d];
        const DescInfo inf = ws.info[d];
        s1::EmbedView a;
        a.cover = D.cover;
        a.stego = D.stego;
        a.msg = D.msg;
        a.n_bytes = inf.n_bytes;
        a.t_bytes = inf.t_bytes;
        a.slen = inf.len;
        a.header = (inf.bits & kHeader) ? 1u : 0u;
        a.nbits = inf.nbits;
        a.msg_even = (inf.bits & kMsgEven) ? 1u : 0u;
        a.pad = 0;
        const uint64_t b0 = lt * tile_bytes;
        const uint64_t b1 = b0 + tile_bytes < inf.n_bytes ? b0 + tile_bytes : inf.n_bytes;
        if (inf.bits & kVec) {
            s1::embed_vec_range<V, STATS>(a, (b0 >> 4) + threadIdx.x, b1 >> 4,
                                          (uint64_t)blockDim.x * V, changed, sse);
            if (b1 == inf.n_bytes)
                s1::embed_tail<STATS>(a, changed, sse);
        } else {
            s1::embed_bytes_range<STATS>(a, (b0 >> 3) + threadIdx.x, (b1 + 7) >> 3, blockDim.x,
                                         changed, sse);
        }
    });
    if (STATS)
        flush_stats(changed, sse, stat_d < n ? results + stat_d : nullptr);
}

template <int V>
__global__ void __launch_bounds__(512) persist_extract(const stego_desc *descs, uint32_t n,
                                                       WsView ws, uint32_t tile_bytes)
{
    grid_dependency_wait(); // launched dependent: nothing is touched before
    allow_dependents();
    claim_loop(ws.start, ws.head->total, &ws.head->counter, n,
               [&](uint32_t d, unsigned long long lt) {
        const stego_desc &D = descs[d];
        const DescInfo inf = ws.info[d];
        s1::ExtractView x;
        x.st = D.cover;
        x.msg = D.msg;
        x.len = inf.len;
        x.base = (inf.bits & kHeader) ? 32u : 0u;
        x.msg_even = (inf.bits & kMsgEven) ? 1u : 0u;
        x.pad = 0;
        const uint64_t b0 = lt * tile_bytes;
        const uint64_t b1 = b0 + tile_bytes < inf.n_bytes ? b0 + tile_bytes : inf.n_bytes;
        if (inf.bits & kVec) {
            s1::extract_vec_range<V>(x, (b0 >> 4) + threadIdx.x, b1 >> 4, (uint64_t)blockDim.x * V);
            if (b1 == inf.n_bytes && (x.len & 1u) && threadIdx.x == 0)
                s1::extract_one(x, x.len - 1);
        } else {
            s1::extract_bytes_range(x, (b0 >> 3) + threadIdx.x, b1 >> 3, blockDim.x);
        }
    });
}

// One-bit stream covers whose buffers are not 16-byte aligned, in their own
// tile space and kernels, so that the aligned kernels keep their register
// budget (calling these routines from them raised persist_embed<4, true>
// from 80 to 94 registers and persist_extract<4> from 39 to 64).  A tile is
// per_tile aligned stego vectors (embed) or message byte pairs (extract);
// the routines are the single-cover kernels' (same misalignment: vectors
// after a scalar head, two per thread and round; different misalignments:
// each stego vector joined from the two aligned cover vectors around its
// bytes, the second passed from the next lane, blocks of 4 x 32 vectors per
// warp; extraction: aligned stego vectors reduced to their LSBs, a pair's
// bits cut from two lanes', four per thread).
constexpr int kMisV = 2, kMisFunnelV = 4, kMisXV = 4;

template <int Q, bool STATS>
__device__ __forceinline__ void mis_funnel(const s1::EmbedView &a, uint32_t h, uint32_t sel,
                                           uint64_t j0, uint64_t j1, unsigned long long &changed,
                                           unsigned long long &sse)
{
    s1::embed_funnel_warp<Q, STATS, kMisFunnelV>(a, h, sel, j0, j1, threadIdx.x >> 5,
                                                 blockDim.x >> 5, changed, sse);
}

// One tile of a misaligned stream cover (the CTA's threads together).
template <bool STATS>
__device__ __forceinline__ void mis_embed_tile(const stego_desc &D, const DescInfo &inf,
                                               unsigned long long lt,
                                               unsigned long long &changed,
                                               unsigned long long &sse)
{
        s1::EmbedView a;
        a.cover = D.cover;
        a.stego = D.stego;
        a.msg = D.msg;
        a.n_bytes = inf.n_bytes;
        a.t_bytes = inf.t_bytes;
        a.slen = inf.len;
        a.header = (inf.bits & kHeader) ? 1u : 0u;
        a.nbits = inf.nbits;
        a.msg_even = (inf.bits & kMsgEven) ? 1u : 0u;
        a.pad = 0;
        const uint32_t h = inf.W;
        const uint64_t nvb = (inf.n_bytes - h) >> 4;
        const uint64_t j0 = lt * inf.per_tile;
        const uint64_t j1 = j0 + inf.per_tile < nvb ? j0 + inf.per_tile : nvb;
        if (inf.bits & kFunnel) {
            switch (inf.channels) {
            case 0: mis_funnel<0, STATS>(a, h, inf.H, j0, j1, changed, sse); break;
            case 1: mis_funnel<1, STATS>(a, h, inf.H, j0, j1, changed, sse); break;
            case 2: mis_funnel<2, STATS>(a, h, inf.H, j0, j1, changed, sse); break;
            default: mis_funnel<3, STATS>(a, h, inf.H, j0, j1, changed, sse); break;
            }
        } else {
            s1::embed_shift_range<kMisV, STATS>(a, h, j0 + threadIdx.x, j1,
                                                (uint64_t)blockDim.x * kMisV, changed, sse);
        }
        // the h head bytes with the first tile, the tail (under one vector)
        // with the last, one byte per thread
        const uint32_t tail = (uint32_t)(inf.n_bytes - h - (nvb << 4));
        uint64_t k = ~0ull;
        if (lt == 0 && threadIdx.x < h)
            k = threadIdx.x;
        else if (j1 == nvb && threadIdx.x >= 16 && threadIdx.x - 16 < tail)
            k = h + (nvb << 4) + (threadIdx.x - 16);
        if (k != ~0ull) {
            const uint32_t sb = k < a.t_bytes ? s1::stream_byte(a, k >> 3) : 0u;
            s1::embed_one<STATS>(a, k, sb, changed, sse);
        }
}

__device__ __forceinline__ void mis_extract_tile(const stego_desc &D, const DescInfo &inf,
                                                 unsigned long long lt)
{
        s1::ExtractView x;
        x.st = D.cover;
        x.msg = D.msg;
        x.len = inf.len;
        x.base = (inf.bits & kHeader) ? 32u : 0u;
        x.msg_even = (inf.bits & kMsgEven) ? 1u : 0u;
        x.pad = 0;
        const uint64_t np = inf.len >> 1;
        const uint64_t p0 = lt * inf.per_tile;
        const uint64_t p1 = p0 + inf.per_tile < np ? p0 + inf.per_tile : np;
        s1::extract_shift_lsb<kMisXV>(x, D.cover_bytes, p0, p1, threadIdx.x >> 5,
                                      blockDim.x >> 5);
        if (p1 == np && (x.len & 1u) && threadIdx.x == 0)
            s1::extract_one(x, x.len - 1);
}

// The misaligned stream tiles' own persistent kernels, with register
// budgets of their own (inside the paper layout's kernel the embed ran at
// 0.69 of the HBM peak on 4096 covers).  The embed runs three CTAs of 256
// threads per SM at 80 registers: with one cover load per stego vector
// (the funnel's second vector shuffled from the next lane) four vectors per
// lane fit, 48 KiB of cover in flight per SM; on the 4096-cover batch at
// offsets 1..15 that took the embed from 2.95 to 2.67 ms (0.83 to 0.92 of
// the peak; the two-load form at two vectors: two CTAs of 512 threads at
// 64 registers; the shuffled form at two vectors or at four in two CTAs of
// 512 threads: 2.92-2.97 ms).  The extract runs CTAs of 128 threads (48
// registers, ten per SM), a 64 KiB tile being eight rounds of their warps:
// on the same batch 0.84 ms with 256 threads, 0.75 ms with 128, as fast as
// the aligned batch in the same launch shape (512 threads: 0.87 against
// 0.76 of the peak with 256; eight vectors per lane: 0.75-0.77 ms).
constexpr int kMisEmbedThreads = 256, kMisEmbedMinCtas = 3, kMisExtractThreads = 128;
template <bool STATS>
__global__ void __launch_bounds__(kMisEmbedThreads, kMisEmbedMinCtas)
    persist_mis_embed(const stego_desc *descs, uint32_t n, stego_result *results, WsView ws)
{
    grid_dependency_wait(); // launched dependent: nothing is touched before
    allow_dependents();
    unsigned long long changed = 0, sse = 0;
    uint32_t stat_d = 0xFFFFFFFFu;
    claim_loop(ws.start_m, ws.head->total_m, &ws.head->counter_m, n,
               [&](uint32_t d, unsigned long long lt) {
        if (STATS && d != stat_d) {
            flush_stats(changed, sse, stat_d < n ? results + stat_d : nullptr);
            stat_d = d;
        }
        mis_embed_tile<STATS>(descs[d], ws.info[d], lt, changed, sse);
    });
    if (STATS)
        flush_stats(changed, sse, stat_d < n ? results + stat_d : nullptr);
}

__global__ void __launch_bounds__(kMisExtractThreads)
    persist_mis_extract(const stego_desc *descs, uint32_t n, WsView ws)
{
    grid_dependency_wait(); // launched dependent: nothing is touched before
    allow_dependents();
    claim_loop(ws.start_m, ws.head->total_m, &ws.head->counter_m, n,
               [&](uint32_t d, unsigned long long lt) {
        mis_extract_tile(descs[d], ws.info[d], lt);
    });
}

// The paper layout's own persistent kernels (a separate register budget from
// the stream kernels): tiles of units, rows or runs, claimed like above.
// Capped at 80 registers for three CTAs per SM: on 600 video frames the
// embed with statistics went from 1.47 to 1.32 ms and the extract from 0.54
// to 0.48 ms, although the statistics variant spills (120 bytes).
template <bool STATS>
__global__ void __launch_bounds__(kP2Threads, 3) persist_p2_embed(const stego_desc *descs, uint32_t n,
                                                        stego_result *results, WsView ws)
{
    grid_dependency_wait(); // launched dependent: nothing is touched before
    allow_dependents();
    unsigned long long changed = 0, sse = 0;
    uint32_t stat_d = 0xFFFFFFFFu;
    claim_loop(ws.start_p, ws.head->total_p, &ws.head->counter_p, n,
               [&](uint32_t d, unsigned long long lt) {
        if (STATS && d != stat_d) {
            flush_stats(changed, sse, stat_d < n ? results + stat_d : nullptr);
            stat_d = d;
        }
        paper_embed_tile<STATS>(descs[d], ws.info[d], lt, changed, sse);
    });
    if (STATS)
        flush_stats(changed, sse, stat_d < n ? results + stat_d : nullptr);
}

__global__ void __launch_bounds__(kP2Threads, 3) persist_p2_extract(const stego_desc *descs, uint32_t n,
                                                          WsView ws)
{
    grid_dependency_wait(); // launched dependent: nothing is touched before
    allow_dependents();
    claim_loop(ws.start_p, ws.head->total_p, &ws.head->counter_p, n,
               [&](uint32_t d, unsigned long long lt) {
        paper_extract_tile(descs[d], ws.info[d], lt);
    });
}

template <bool EMBED>
const void *persist_kernel(int vec, bool stats)
{
    if (EMBED) {
        switch (vec) {
        case 1: return stats ? (const void *)persist_embed<1, true> : (const void *)persist_embed<1, false>;
        case 2: return stats ? (const void *)persist_embed<2, true> : (const void *)persist_embed<2, false>;
        case 8: return stats ? (const void *)persist_embed<8, true> : (const void *)persist_embed<8, false>;
        default: return stats ? (const void *)persist_embed<4, true> : (const void *)persist_embed<4, false>;
        }
    }
    switch (vec) {
    case 1: return (const void *)persist_extract<1>;
    case 2: return (const void *)persist_extract<2>;
    case 8: return (const void *)persist_extract<8>;
    default: return (const void *)persist_extract<4>;
    }
}

uint64_t workspace_bytes(uint32_t n) { return info_off(n) + sizeof(DescInfo) * (uint64_t)n; }

template <bool EMBED>
int batched(const stego_desc *d_descs, uint32_t n, stego_result *d_results, uint32_t flags,
            const stego_tune *tune, void *d_ws, uint64_t ws_bytes, void *stream)
{
    if (flags & ~(uint32_t)STEGO_FUSE_STATS)
        return STEGO_E_INVAL;
    if (!EMBED && (flags & STEGO_FUSE_STATS))
        return STEGO_E_INVAL;
    if (tune && !tune_ok(tune))
        return STEGO_E_INVAL;
    if (n == 0)
        return STEGO_OK;
    if (!d_descs || !d_results || !d_ws)
        return STEGO_E_INVAL;
    if (((uintptr_t)d_descs & 7u) || ((uintptr_t)d_results & 7u) || ((uintptr_t)d_ws & 15u))
        return STEGO_E_INVAL;
    if (ws_bytes < workspace_bytes(n))
        return STEGO_E_NOMEM;
    cudaStream_t s = (cudaStream_t)stream;
    const Shape sh = shape_for(EMBED ? STEGO_OP_EMBED_BATCHED : STEGO_OP_EXTRACT_BATCHED, tune);
    const uint32_t tile = sh.tile_bytes;
    WsView ws = ws_view(d_ws, n);

    const int prep_threads = 256;
    int prep_grid = (int)((n + prep_threads - 1) / prep_threads);
    const int prep_cap = sm_count() * 8;
    if (prep_grid > prep_cap)
        prep_grid = prep_cap;
    cudaError_t e;
    {
        uint32_t tile_arg = tile;
        void *args[] = {(void *)&d_descs, &n, &d_results, &ws, &tile_arg};
        e = launch_dependent(EMBED ? (const void *)prep_embed : (const void *)prep_extract,
                             dim3(prep_grid), dim3(prep_threads), args, 0, s);
    }
    if (e != cudaSuccess)
        return STEGO_E_CUDA;
    {
        void *args[] = {&ws, &n};
        e = launch_dependent((const void *)scan_tiles, dim3(1), dim3(kScanThreads), args, 0, s);
    }
    if (e != cudaSuccess)
        return STEGO_E_CUDA;

    const bool stats = (flags & STEGO_FUSE_STATS) != 0;
    const void *k = persist_kernel<EMBED>(sh.vec, stats);
    // the tile count lives on the device: launch the full persistent grid
    const int grid = persistent_grid(k, sh.threads, 0, sh.ctas_per_sm, ~0ull >> 1, 1);
    if (EMBED) {
        void *args[] = {(void *)&d_descs, &n, &d_results, &ws, (void *)&tile};
        e = launch_dependent(k, dim3(grid), dim3(sh.threads), args, 0, s);
    } else {
        void *args[] = {(void *)&d_descs, &n, &ws, (void *)&tile};
        e = launch_dependent(k, dim3(grid), dim3(sh.threads), args, 0, s);
    }
    if (e != cudaSuccess)
        return STEGO_E_CUDA;
    // misaligned stream tiles (count on the device; an empty set exits at once)
    {
        const int mis_threads = EMBED ? kMisEmbedThreads : kMisExtractThreads;
        const void *km = EMBED ? (stats ? (const void *)persist_mis_embed<true>
                                        : (const void *)persist_mis_embed<false>)
                               : (const void *)persist_mis_extract;
        const int gridm = persistent_grid(km, mis_threads, 0, 0, ~0ull >> 1, 1);
        if (EMBED) {
            void *args[] = {(void *)&d_descs, &n, &d_results, &ws};
            e = launch_dependent(km, dim3(gridm), dim3(mis_threads), args, 0, s);
        } else {
            void *args[] = {(void *)&d_descs, &n, &ws};
            e = launch_dependent(km, dim3(gridm), dim3(mis_threads), args, 0, s);
        }
    }
    if (e != cudaSuccess)
        return STEGO_E_CUDA;
    // paper-layout tiles (their count is on the device; an empty set exits at once)
    const int p2_threads = (int)kP2Threads;
    const void *kp = EMBED ? (stats ? (const void *)persist_p2_embed<true>
                                    : (const void *)persist_p2_embed<false>)
                           : (const void *)persist_p2_extract;
    const int gridp = persistent_grid(kp, p2_threads, 0, 0, ~0ull >> 1, 1);
    if (EMBED) {
        void *args[] = {(void *)&d_descs, &n, &d_results, &ws};
        e = launch_dependent(kp, dim3(gridp), dim3(p2_threads), args, 0, s);
    } else {
        void *args[] = {(void *)&d_descs, &n, &ws};
        e = launch_dependent(kp, dim3(gridp), dim3(p2_threads), args, 0, s);
    }
    return e == cudaSuccess ? STEGO_OK : STEGO_E_CUDA;
}

} // namespace
} // namespace stego

using namespace stego;

struct stego_graph {
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

extern "C" {

uint64_t stego_batched_workspace_bytes(uint32_t n) { return workspace_bytes(n); }

int stego_embed_batched(const stego_desc *d_descs, uint32_t n, stego_result *d_results,
                        uint32_t flags, const stego_tune *tune, void *d_ws, uint64_t ws_bytes,
                        void *stream)
{
    stego::Trace trace_("stego_embed_batched");
    return batched<true>(d_descs, n, d_results, flags, tune, d_ws, ws_bytes, stream);
}

int stego_extract_batched(const stego_desc *d_descs, uint32_t n, stego_result *d_results,
                          uint32_t flags, const stego_tune *tune, void *d_ws, uint64_t ws_bytes,
                          void *stream)
{
    stego::Trace trace_("stego_extract_batched");
    return batched<false>(d_descs, n, d_results, flags, tune, d_ws, ws_bytes, stream);
}

int stego_graph_capture_batched(int op, const stego_desc *d_descs, uint32_t n,
                                stego_result *d_results, uint32_t flags, const stego_tune *tune,
                                void *d_ws, uint64_t ws_bytes, stego_graph **out)
{
    stego::Trace trace_("stego_graph_capture_batched");
    if (!out || (op != STEGO_OP_EMBED_BATCHED && op != STEGO_OP_EXTRACT_BATCHED))
        return STEGO_E_INVAL;
    *out = nullptr;
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
        return STEGO_E_CUDA;
    int st = STEGO_OK;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaStreamDestroy(s);
        return STEGO_E_CUDA;
    }
    if (op == STEGO_OP_EMBED_BATCHED)
        st = stego_embed_batched(d_descs, n, d_results, flags, tune, d_ws, ws_bytes, s);
    else
        st = stego_extract_batched(d_descs, n, d_results, flags, tune, d_ws, ws_bytes, s);
    const cudaError_t ee = cudaStreamEndCapture(s, &g);
    cudaStreamDestroy(s);
    if (st != STEGO_OK) {
        if (g)
            cudaGraphDestroy(g);
        return st;
    }
    if (ee != cudaSuccess || !g)
        return STEGO_E_CUDA;
    cudaGraphExec_t ex = nullptr;
    if (cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) {
        cudaGraphDestroy(g);
        return STEGO_E_CUDA;
    }
    stego_graph *h = new stego_graph;
    h->graph = g;
    h->exec = ex;
    *out = h;
    return STEGO_OK;
}

int stego_graph_launch(stego_graph *g, void *stream)
{
    if (!g)
        return STEGO_E_INVAL;
    return cudaGraphLaunch(g->exec, (cudaStream_t)stream) == cudaSuccess ? STEGO_OK : STEGO_E_CUDA;
}

int stego_graph_destroy(stego_graph *g)
{
    if (!g)
        return STEGO_OK;
    cudaGraphExecDestroy(g->exec);
    cudaGraphDestroy(g->graph);
    delete g;
    return STEGO_OK;
}

} // extern "C"

// ---------------------------------------------------------------------------
// Batched embed for callers that cannot allocate device memory
// ---------------------------------------------------------------------------
// Some callers cannot call cudaMalloc at all: a host program with no device
// allocator of its own, or one that may not add cudaMalloc's implicit device
// synchronisation to its per-request path.  They still own descriptors,
// covers, messages and results; only the batched call's scratch (tile
// counter, tile offsets, per-cover sizes) moves into this file-scope array,
// sized for STEGO_NOALLOC_MAX_DESCS covers.  Every GPU that loads the library
// holds it until the process exits.

namespace {

constexpr uint32_t kNoAllocMaxDescs = STEGO_NOALLOC_MAX_DESCS;
constexpr uint64_t kNoAllocBytes =
    stego::info_off(kNoAllocMaxDescs) + sizeof(stego::DescInfo) * (uint64_t)kNoAllocMaxDescs;
constexpr int kNoAllocDevices = 64;

std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kNoAllocDevices];              // device address of the array, per device
unsigned long long g_noalloc_ctx[kNoAllocDevices]; // the context that address belongs to

} // namespace

// In host code this name is only a host-side stand-in for the device array:
// the kernels get the address that cudaGetSymbolAddress returns.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {

// Device address of the scratch array on the current device, looked up once
// per device with that device current, and again after the device was reset
// (its context changed: the module, and with it the array, was loaded anew).
int noalloc_scratch(void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return STEGO_E_CUDA;
    if (dev < 0 || dev >= kNoAllocDevices)
        return STEGO_E_INVAL;
    const unsigned long long ctx = stego::context_id();
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev] || !ctx || g_noalloc_ctx[dev] != ctx) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return STEGO_E_CUDA;
        g_noalloc_ptr[dev] = p;
        g_noalloc_ctx[dev] = ctx;
    }
    *out = g_noalloc_ptr[dev];
    return STEGO_OK;
}

} // namespace

extern "C" int stego_embed_batched_noalloc(const stego_desc *d_descs, uint32_t n,
                                           stego_result *d_results, uint32_t flags,
                                           const stego_tune *tune, void *stream)
{
    stego::Trace trace_("stego_embed_batched_noalloc");
    // argument errors first, as stego_embed_batched reports them
    if (flags & ~(uint32_t)STEGO_FUSE_STATS)
        return STEGO_E_INVAL;
    if (tune && !stego::tune_ok(tune))
        return STEGO_E_INVAL;
    if (n > kNoAllocMaxDescs)
        return STEGO_E_NOMEM;
    if (n == 0)
        return STEGO_OK;
    void *ws = nullptr;
    const int st = noalloc_scratch(&ws);
    if (st != STEGO_OK)
        return st;
    // the prep and scan launches rewrite every scratch word the persistent
    // kernel reads, so the previous call's contents need no clearing
    return stego::batched<true>(d_descs, n, d_results, flags, tune, ws, kNoAllocBytes, stream);
}
