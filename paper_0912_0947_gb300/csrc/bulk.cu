// bulk.cu -- shared-memory staged variants of the one-bit stream kernels
// (the Section VI substitution and the Section VII extraction, one bit per
// cover byte in memory order, as in stream1.cu).
//
// Tiles of the cover (embed) or of the stego's carrying bytes (extract) move
// from HBM into a ring of shared-memory stages with one-dimensional bulk
// asynchronous copies: one thread issues `cp.async.bulk` for a whole tile and
// the copy counts its bytes on the stage's mbarrier, so a CTA keeps several
// tiles in flight with one instruction each, where the register kernels need
// one 128-bit load per thread and vector.  The threads transform a landed
// tile; the embed writes it back from registers with 128-bit streaming
// stores (or, with kBulkStore, in shared memory followed by one bulk store
// per tile, bulk-group completion).  Message bytes (1/8 of the cover
// traffic) are read with 16-bit loads one tile ahead.
//
// Shape: threads per CTA, V vectors per thread per tile (tile = threads * 16
// * V bytes), stages = ring bytes / tile, 2..8 stages.  Tiles are dealt to a
// persistent grid round-robin.
//
// Every wait is bounded (one second of %globaltimer).  A CTA whose wait runs
// out stops, waits (bounded again) for the copies it still has in flight and
// for its bulk stores, writes STEGO_E_TIMEOUT into the result and returns.
// stego_test_bounded_wait shortens the bound and can make every CTA's first
// wait run out (each stage's barrier then expects one arrival more than the
// pipeline gives; the CTA gives it while draining), so that the timeout path
// runs on demand without any fault.
#include <atomic>
#include <mutex>

#include "s1_device.cuh"

namespace stego {
namespace {

constexpr int kMaxStages = 8;
constexpr uint32_t kMaxRingBytes = 192u * 1024u;
constexpr uint64_t kWaitNs = 1000000000ull;
// Process-wide settings of stego_test_bounded_wait, read at each launch.
std::atomic<uint64_t> g_wait_ns{kWaitNs};
std::atomic<uint32_t> g_withhold{0};
// Measured on the 201 MB full-capacity embed and extract (same box, best
// shape of each): the embed is fastest with loads without a cache hint and
// stores from registers (70.9 us; 72.7 us with evict-first loads, 72.7 us
// with bulk stores, 74.8 us with both), the extract with evict-first loads
// (36.4-36.9 us against 38.9 us without).  The register kernels take
// 66.9-68.6 us and 35.8-36.6 us on the same box.
constexpr bool kBulkStore = false;
constexpr bool kEmbedEvictFirst = false;
constexpr bool kExtractEvictFirst = true;

// ---------------------------------------------------------------------------
// mbarrier and bulk-copy primitives (PTX ISA: mbarrier, cp.async.bulk)
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

// Makes the initialised barriers visible to the asynchronous proxy.
__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// One plain arrival.
__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// One arrival that also announces `bytes` of transaction count.
__device__ __forceinline__ void mbar_arrive_expect(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t done;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(done)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    return done != 0;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for the phase with the given parity to complete; false after
// limit_ns without completion.
__device__ __noinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint64_t limit_ns)
{
    if (mbar_try_wait(bar, parity))
        return true;
    const uint64_t t0 = global_ns();
    for (uint32_t n = 1;; ++n) {
        if (mbar_try_wait(bar, parity))
            return true;
        if ((n & 63u) == 0 && global_ns() - t0 > limit_ns)
            return false;
    }
}

// L2 policy for data touched once.
__device__ __forceinline__ uint64_t evict_first_policy()
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// Global -> shared, `bytes` (multiple of 16, both addresses 16-byte aligned)
// counted on `bar`; with `evict_first` the lines get the L2 evict-first
// policy.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes,
                                          uint64_t *bar, bool evict_first)
{
    if (evict_first)
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes"
                     ".L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(smem_u32(dst)),
                     "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(evict_first_policy())
                     : "memory");
    else
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes "
                     "[%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
                     "l"(src), "r"(bytes), "r"(smem_u32(bar))
                     : "memory");
}

// Shared -> global, tracked by bulk groups.
__device__ __forceinline__ void bulk_store(void *dst, const void *src, uint32_t bytes)
{
    if (kEmbedEvictFirst)
        asm volatile("cp.async.bulk.global.shared::cta.bulk_group.L2::cache_hint"
                     " [%0], [%1], %2, %3;" ::"l"(dst),
                     "r"(smem_u32(src)), "r"(bytes), "l"(evict_first_policy())
                     : "memory");
    else
        asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
                     "r"(smem_u32(src)), "r"(bytes)
                     : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

// All but the most recent group have finished reading shared memory.
__device__ __forceinline__ void bulk_wait_read_but_one()
{
    asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
}

// Every group has completed (its writes are performed).
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Orders this thread's shared-memory writes before later bulk copies read them.
__device__ __forceinline__ void fence_async_shared()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ---------------------------------------------------------------------------
// Tile bookkeeping shared by both kernels
// ---------------------------------------------------------------------------

struct Ring {
    uint8_t *base;     // stage s at base + s * tile
    uint64_t *full;    // one barrier per stage
    uint32_t stages;
    uint32_t tile;     // bytes per stage
    const uint8_t *src; // 16-byte aligned source of vector 0
    uint64_t nvec;     // 16-byte vectors to move
    uint64_t tvec;     // vectors per tile
    uint64_t first;    // this CTA's first tile
    uint64_t step;     // tile stride (grid size)
    bool evict_first;  // L2 policy of the loads

    __device__ uint64_t v0(uint64_t i) const { return (first + i * step) * tvec; }
    __device__ uint32_t bytes(uint64_t i) const
    {
        const uint64_t v = v0(i);
        return (uint32_t)((nvec - v < tvec ? nvec - v : tvec) << 4);
    }
    __device__ uint8_t *stage(uint64_t i) const { return base + (uint32_t)(i % stages) * tile; }
    __device__ uint64_t *bar(uint64_t i) const { return full + (uint32_t)(i % stages); }
    __device__ uint32_t parity(uint64_t i) const { return (uint32_t)(i / stages) & 1u; }
    // Called by one thread: the load of this CTA's tile i into its stage.
    __device__ void issue(uint64_t i) const
    {
        const uint32_t b = bytes(i);
        mbar_arrive_expect(bar(i), b);
        bulk_load(stage(i), src + (v0(i) << 4), b, bar(i), evict_first);
    }
};

// Tiles of this CTA when `ntiles` tiles are dealt round-robin.
__device__ __forceinline__ uint64_t local_tiles(uint64_t ntiles)
{
    return blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
}

// After a timeout: wait (bounded by the default limit) for the loads of
// tiles [from, issued), then for the bulk stores, and report the timeout.
// With `withheld`, each of those stages still lacks the arrival its barrier
// was initialised to expect: it is given here, so the phase completes once
// the copy's bytes have landed.
__device__ void drain_after_timeout(const Ring &r, uint64_t from, uint64_t issued,
                                    stego_result *res, bool withheld)
{
    if (withheld)
        for (uint64_t i = from; i < issued; ++i)
            mbar_arrive(r.bar(i));
    for (uint64_t i = from; i < issued; ++i)
        mbar_wait(r.bar(i), r.parity(i), kWaitNs);
    bulk_wait_all();
    if (res)
        *(volatile int32_t *)&res->status = STEGO_E_TIMEOUT;
}

// ---------------------------------------------------------------------------
// Embed
// ---------------------------------------------------------------------------

struct BulkEmbedArgs {
    s1::EmbedView a;
    stego_result *res;
    uint64_t res_msg_bytes;
    StatSlot *slot;
    uint32_t stages;
    uint32_t withhold; // barriers expect one arrival the pipeline never gives
    uint64_t wait_ns;  // bound of the pipeline's waits
};

// Stream pairs of this thread's vectors of tile i (0 past the stream).
template <int V>
__device__ __forceinline__ void tile_pairs(const s1::EmbedView &a, const Ring &r, uint64_t i,
                                           uint32_t (&p)[V])
{
    const uint64_t v0 = r.v0(i);
#pragma unroll
    for (int u = 0; u < V; ++u) {
        const uint64_t v = v0 + threadIdx.x + (uint64_t)u * blockDim.x;
        p[u] = (v < r.nvec && (v << 4) < a.t_bytes) ? s1::stream_pair(a, v << 1) : 0u;
    }
}

template <int V, bool STATS>
__global__ void __launch_bounds__(512) embed_bulk(BulkEmbedArgs e)
{
    grid_dependency_wait(); // launched dependent: nothing is touched before
    allow_dependents();
    extern __shared__ __align__(128) uint8_t ring_mem[];
    __shared__ __align__(8) uint64_t full[kMaxStages];
    const s1::EmbedView &a = e.a;
    unsigned long long changed = 0, sse = 0;
    if (e.res && blockIdx.x == 0 && threadIdx.x == 0) {
        e.res->msg_bytes = e.res_msg_bytes;
        e.res->status = STEGO_OK;
        e.res->reserved = 0;
        if (!STATS) {
            e.res->changed = 0;
            e.res->sse = 0;
        }
    }
    Ring r;
    r.base = ring_mem;
    r.full = full;
    r.stages = e.stages;
    r.tvec = (uint64_t)blockDim.x * V;
    r.tile = (uint32_t)(r.tvec << 4);
    r.src = a.cover;
    r.nvec = a.n_bytes >> 4;
    r.first = blockIdx.x;
    r.step = gridDim.x;
    r.evict_first = kEmbedEvictFirst;
    const uint64_t nl = local_tiles((r.nvec + r.tvec - 1) / r.tvec);
    if (threadIdx.x == 0) {
        for (uint32_t s = 0; s < r.stages; ++s)
            mbar_init(&full[s], e.withhold ? 2u : 1u);
        mbar_init_fence();
    }
    __syncthreads();
    uint64_t issued = 0;
    if (threadIdx.x == 0)
        for (; issued < nl && issued < r.stages; ++issued)
            r.issue(issued);
    uint32_t p[V];
    if (nl)
        tile_pairs<V>(a, r, 0, p);
    uint4 *dst = reinterpret_cast<uint4 *>(a.stego);
    uint64_t i = 0;
    bool failed = false;
    for (; i < nl; ++i) {
        uint32_t pc[V];
#pragma unroll
        for (int u = 0; u < V; ++u)
            pc[u] = p[u];
        if (i + 1 < nl)
            tile_pairs<V>(a, r, i + 1, p); // in flight while this tile lands
        const bool ok = mbar_wait(r.bar(i), r.parity(i), e.wait_ns);
        const uint64_t v0 = r.v0(i);
        if (ok) {
            uint4 *buf = reinterpret_cast<uint4 *>(r.stage(i));
            uint32_t n = 0;
#pragma unroll
            for (int u = 0; u < V; ++u) {
                const uint32_t j = threadIdx.x + u * blockDim.x;
                const uint64_t v = v0 + j;
                if (v < r.nvec) {
                    const uint4 o = s1::embed_vec16<STATS>(a, v, buf[j], pc[u], n);
                    if (kBulkStore)
                        buf[j] = o;
                    else
                        __stcs(dst + v, o);
                }
            }
            if (STATS) {
                changed += n;
                sse += n;
            }
            if (kBulkStore)
                fence_async_shared();
        }
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        if (threadIdx.x == 0) {
            if (kBulkStore) {
                bulk_store(a.stego + (v0 << 4), r.stage(i), r.bytes(i));
                bulk_commit();
                // refill the stage of tile i-1 once its store has read it
                if (i >= 1 && issued < nl) {
                    bulk_wait_read_but_one();
                    r.issue(issued++);
                }
            } else if (issued < nl) {
                r.issue(issued++); // every thread has read stage i
            }
        }
    }
    if (threadIdx.x == 0) {
        if (failed)
            drain_after_timeout(r, i, issued, e.res, e.withhold != 0);
        else
            bulk_wait_all();
    }
    if (blockIdx.x == 0 && !failed) // `failed` is the same in every thread
        s1::embed_tail<STATS>(a, changed, sse);
    if (STATS)
        block_stats(changed, sse, e.res, e.slot);
}

// ---------------------------------------------------------------------------
// Extract
// ---------------------------------------------------------------------------

struct BulkExtractArgs {
    s1::ExtractArgs x;
    uint32_t stages;
    uint32_t withhold; // as in BulkEmbedArgs
    uint64_t wait_ns;
};

template <int V>
__global__ void __launch_bounds__(512) extract_bulk(BulkExtractArgs e)
{
    grid_dependency_wait(); // launched dependent: nothing is touched before
    allow_dependents();
    extern __shared__ __align__(128) uint8_t ring_mem[];
    __shared__ __align__(8) uint64_t full[kMaxStages];
    s1::ExtractView x;
    if (s1::extract_prologue(e.x, x) != STEGO_OK)
        return;
    Ring r;
    r.base = ring_mem;
    r.full = full;
    r.stages = e.stages;
    r.tvec = (uint64_t)blockDim.x * V;
    r.tile = (uint32_t)(r.tvec << 4);
    r.src = x.st + x.base;
    r.nvec = x.len >> 1; // vector v -> message bytes 2v, 2v+1
    r.first = blockIdx.x;
    r.step = gridDim.x;
    r.evict_first = kExtractEvictFirst;
    const uint64_t nl = local_tiles((r.nvec + r.tvec - 1) / r.tvec);
    if (threadIdx.x == 0) {
        for (uint32_t s = 0; s < r.stages; ++s)
            mbar_init(&full[s], e.withhold ? 2u : 1u);
        mbar_init_fence();
    }
    __syncthreads();
    uint64_t issued = 0;
    if (threadIdx.x == 0)
        for (; issued < nl && issued < r.stages; ++issued)
            r.issue(issued);
    uint64_t i = 0;
    bool failed = false;
    for (; i < nl; ++i) {
        const bool ok = mbar_wait(r.bar(i), r.parity(i), e.wait_ns);
        if (ok) {
            const uint4 *buf = reinterpret_cast<const uint4 *>(r.stage(i));
            const uint64_t v0 = r.v0(i);
#pragma unroll
            for (int u = 0; u < V; ++u) {
                const uint32_t j = threadIdx.x + u * blockDim.x;
                const uint64_t v = v0 + j;
                if (v < r.nvec) {
                    const uint32_t pair = s1::gather16(buf[j]);
                    if (x.msg_even) {
                        *reinterpret_cast<unsigned short *>(x.msg + 2 * v) = (unsigned short)pair;
                    } else {
                        x.msg[2 * v] = (uint8_t)pair;
                        x.msg[2 * v + 1] = (uint8_t)(pair >> 8);
                    }
                }
            }
        }
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        if (threadIdx.x == 0 && issued < nl)
            r.issue(issued++); // every thread has read stage i
    }
    if (threadIdx.x == 0 && failed)
        drain_after_timeout(r, i, issued, e.x.res, e.withhold != 0);
    if ((x.len & 1u) && blockIdx.x == 0 && threadIdx.x == 0 && !failed)
        s1::extract_one(x, x.len - 1);
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

int clamp_v(int v) { return (v == 1 || v == 2 || v == 8) ? v : 4; }

std::mutex g_attr_mu;
const void *g_attr_done[64][32]; // per device: kernels whose smem limit is raised
int g_attr_n[64];
unsigned long long g_attr_ctx[64]; // the context the raised limits belong to

// Raises the kernel's dynamic shared memory limit to kMaxRingBytes once per
// device (again after a device reset, which gives the device a new context).
cudaError_t allow_ring(const void *k)
{
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64)
        dev = 0;
    const unsigned long long ctx = context_id();
    std::lock_guard<std::mutex> lk(g_attr_mu);
    if (!ctx || g_attr_ctx[dev] != ctx) {
        g_attr_n[dev] = 0;
        g_attr_ctx[dev] = ctx;
    }
    for (int i = 0; i < g_attr_n[dev]; ++i)
        if (g_attr_done[dev][i] == k)
            return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kMaxRingBytes);
    if (e == cudaSuccess && g_attr_n[dev] < 32)
        g_attr_done[dev][g_attr_n[dev]++] = k;
    return e;
}

template <bool STATS>
const void *embed_kernel(int v)
{
    switch (v) {
    case 1: return (const void *)embed_bulk<1, STATS>;
    case 2: return (const void *)embed_bulk<2, STATS>;
    case 8: return (const void *)embed_bulk<8, STATS>;
    default: return (const void *)embed_bulk<4, STATS>;
    }
}

const void *extract_kernel(int v)
{
    switch (v) {
    case 1: return (const void *)extract_bulk<1>;
    case 2: return (const void *)extract_bulk<2>;
    case 8: return (const void *)extract_bulk<8>;
    default: return (const void *)extract_bulk<4>;
    }
}

} // namespace

uint32_t bulk_stages(const Shape &sh)
{
    if (!sh.tile_bytes)
        return 0;
    const uint64_t tile = (uint64_t)sh.threads * 16u * (uint64_t)clamp_v(sh.vec);
    uint64_t st = sh.tile_bytes / tile;
    if (st > (uint64_t)kMaxStages)
        st = kMaxStages;
    while (st >= 2 && st * tile > kMaxRingBytes)
        --st;
    return st >= 2 ? (uint32_t)st : 0u;
}

cudaError_t s1_embed_bulk(const uint8_t *cover, uint8_t *stego, uint64_t n_bytes,
                          uint64_t t_bytes, const uint8_t *msg, uint64_t slen, bool header,
                          uint32_t nbits, bool stats, stego_result *res, uint64_t res_msg_bytes,
                          const Shape &sh, cudaStream_t s, StatSlot *slot)
{
    BulkEmbedArgs e;
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
    e.stages = bulk_stages(sh);
    e.withhold = g_withhold.load(std::memory_order_relaxed);
    e.wait_ns = g_wait_ns.load(std::memory_order_relaxed);
    const int v = clamp_v(sh.vec);
    const void *k = stats ? embed_kernel<true>(v) : embed_kernel<false>(v);
    cudaError_t err = allow_ring(k);
    if (err != cudaSuccess)
        return err;
    const size_t ring = (size_t)e.stages * sh.threads * 16u * v;
    const uint64_t tvec = (uint64_t)sh.threads * v;
    const uint64_t ntiles = ((n_bytes >> 4) + tvec - 1) / tvec;
    const int grid = persistent_grid(k, sh.threads, ring, sh.ctas_per_sm, ntiles ? ntiles : 1, 1);
    void *args[] = {&e};
    return launch_dependent(k, dim3(grid), dim3(sh.threads), args, ring, s);
}

cudaError_t s1_extract_bulk(const uint8_t *st, uint64_t C, uint8_t *msg, uint64_t cap,
                            uint64_t raw_len, bool header, stego_result *res, const Shape &sh,
                            cudaStream_t s)
{
    BulkExtractArgs e;
    e.x.st = st;
    e.x.C = C;
    e.x.msg = msg;
    e.x.cap = cap;
    e.x.raw_len = raw_len;
    e.x.header = header ? 1u : 0u;
    e.x.msg_even = ((uintptr_t)msg & 1u) == 0;
    e.x.res = res;
    e.stages = bulk_stages(sh);
    e.withhold = g_withhold.load(std::memory_order_relaxed);
    e.wait_ns = g_wait_ns.load(std::memory_order_relaxed);
    uint64_t max_len = raw_len;
    if (header) {
        const uint64_t fit = C >= 32 ? (C - 32) / 8 : 0;
        max_len = fit < cap ? fit : cap;
    }
    e.x.max_vec = max_len >> 1;
    const int v = clamp_v(sh.vec);
    const void *k = extract_kernel(v);
    cudaError_t err = allow_ring(k);
    if (err != cudaSuccess)
        return err;
    const size_t ring = (size_t)e.stages * sh.threads * 16u * v;
    const uint64_t tvec = (uint64_t)sh.threads * v;
    const uint64_t ntiles = ((max_len >> 1) + tvec - 1) / tvec;
    const int grid = persistent_grid(k, sh.threads, ring, sh.ctas_per_sm, ntiles ? ntiles : 1, 1);
    void *args[] = {&e};
    return launch_dependent(k, dim3(grid), dim3(sh.threads), args, ring, s);
}

} // namespace stego

extern "C" int stego_test_bounded_wait(uint64_t limit_ns, uint32_t withhold_arrival)
{
    if (withhold_arrival > 1u)
        return STEGO_E_INVAL;
    stego::g_wait_ns.store(limit_ns ? limit_ns : stego::kWaitNs, std::memory_order_relaxed);
    stego::g_withhold.store(withhold_arrival, std::memory_order_relaxed);
    return STEGO_OK;
}
