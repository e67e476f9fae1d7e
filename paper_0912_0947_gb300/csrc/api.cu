// api.cu -- the extern "C" entry points of libstego.so (include/stego.h):
// argument validation on the host, launch-shape bookkeeping, and dispatch to
// the kernels of stream1.cu, paper2.cu, stats.cu and batched.cu.
#include <cstring>
#include <mutex>

#include <cuda.h>

#include "internal.cuh"

namespace stego {
namespace {

constexpr int kVersion = 10000; // 1.0.0
constexpr uint64_t kMaxHeaderMsg = 0x1FFFFFFFull; // 8*m must fit 32 bits
constexpr int kMaxDevices = 64;

std::mutex g_mu;
Shape g_shape[STEGO_OP_COUNT] = {
    {512, 4, 0, 0},      // embed
    {128, 4, 0, 0},      // extract
    {256, 4, 0, 0},      // changed
    {256, 4, 0, 65536},  // embed batched
    {256, 4, 0, 65536},  // extract batched
};
int g_sms[kMaxDevices];

// Statistics slots: per device, the streams (by their process-unique
// stream ID, never reused, unlike a destroyed stream's handle) that own slots
// 0..n-1, the device address of the slot array, and the context those
// belong to.
constexpr int kStatSlots = 256;
unsigned long long g_slot_sid[kMaxDevices][kStatSlots];
int g_slot_n[kMaxDevices];
StatSlot *g_slot_base[kMaxDevices];
unsigned long long g_slot_ctx[kMaxDevices];

struct OccEntry {
    const void *kernel;
    int threads;
    int device;
    int blocks;
    size_t smem;
};
constexpr int kOccSlots = 128;
OccEntry g_occ[kOccSlots];
int g_occ_n = 0;

int occupancy(const void *kernel, int threads, size_t smem)
{
    int dev = 0;
    cudaGetDevice(&dev);
    {
        std::lock_guard<std::mutex> lk(g_mu);
        for (int i = 0; i < g_occ_n; ++i)
            if (g_occ[i].kernel == kernel && g_occ[i].threads == threads &&
                g_occ[i].device == dev && g_occ[i].smem == smem)
                return g_occ[i].blocks;
    }
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kernel, threads, smem) !=
            cudaSuccess ||
        blocks < 1)
        blocks = 1;
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_occ_n < kOccSlots)
        g_occ[g_occ_n++] = OccEntry{kernel, threads, dev, blocks, smem};
    return blocks;
}

bool overlap(const void *p, uint64_t np, const void *q, uint64_t nq)
{
    if (np == 0 || nq == 0 || p == nullptr || q == nullptr)
        return false;
    const uintptr_t a = (uintptr_t)p, b = (uintptr_t)q;
    return a < b + nq && b < a + np;
}

bool valid_tune_field_ranges(const stego_tune &t)
{
    if (t.threads && (t.threads % 32u || t.threads < 64u || t.threads > 512u))
        return false;
    if (t.vec_per_thread && !(t.vec_per_thread == 1 || t.vec_per_thread == 2 ||
                              t.vec_per_thread == 4 || t.vec_per_thread == 8))
        return false;
    if (t.ctas_per_sm > 32u)
        return false;
    if (t.tile_bytes && (t.tile_bytes % 4096u || t.tile_bytes < 4096u))
        return false;
    return true;
}

__global__ void write_result_kernel(stego_result *res, uint64_t msg_bytes, int status)
{
    res->changed = 0;
    res->sse = 0;
    res->msg_bytes = msg_bytes;
    res->status = status;
    res->reserved = 0;
}

int cuda_status(cudaError_t e) { return e == cudaSuccess ? STEGO_OK : STEGO_E_CUDA; }

// Driver entry points for the context identity, resolved through the
// runtime so that the library does not link the driver library itself.
using CtxGetCurrentFn = CUresult(CUDAAPI *)(CUcontext *);
using CtxGetIdFn = CUresult(CUDAAPI *)(CUcontext, unsigned long long *);
std::once_flag g_ctx_once;
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;

// An image geometry that describes exactly cover_bytes bytes.
bool geom_ok(const stego_geom *g, uint64_t cover_bytes)
{
    return g && g->channels > 0 && g->plane < g->channels &&
           (uint64_t)g->width * g->height * g->channels == cover_bytes;
}

uint32_t bits_of(uint32_t flags) { return ((flags & STEGO_BITS_MASK) >> 8) + 1u; }

} // namespace

bool tune_ok(const stego_tune *t) { return t && valid_tune_field_ranges(*t); }

unsigned long long context_id()
{
    std::call_once(g_ctx_once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(f);
    });
    if (!g_ctx_get_current || !g_ctx_get_id)
        return 0;
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (g_ctx_get_current(&c) != CUDA_SUCCESS || !c || g_ctx_get_id(c, &id) != CUDA_SUCCESS)
        return 0;
    return id + 1; // 0 stays "unknown"
}

Shape shape_for(int op, const stego_tune *o)
{
    Shape s;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        s = g_shape[op];
    }
    if (o) {
        if (o->threads)
            s.threads = (int)o->threads;
        if (o->vec_per_thread)
            s.vec = (int)o->vec_per_thread;
        if (o->ctas_per_sm)
            s.ctas_per_sm = (int)o->ctas_per_sm;
        if (o->tile_bytes)
            s.tile_bytes = o->tile_bytes;
    }
    return s;
}

int sm_count()
{
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= kMaxDevices)
        dev = 0;
    int n = g_sms[dev];
    if (n == 0) {
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
            n = 1;
        g_sms[dev] = n;
    }
    return n;
}

cudaError_t launch_dependent(const void *kernel, dim3 grid, dim3 block, void **args,
                             size_t smem, cudaStream_t s)
{
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    std::memset(at, 0, sizeof(at));
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, kernel, args);
}

int persistent_grid(const void *kernel, int threads, size_t smem, int ctas_per_sm,
                    uint64_t units, uint64_t units_per_cta)
{
    int per_sm = occupancy(kernel, threads, smem);
    if (ctas_per_sm > 0 && ctas_per_sm < per_sm)
        per_sm = ctas_per_sm;
    const uint64_t cap = (uint64_t)sm_count() * (uint64_t)per_sm;
    uint64_t want = (units + units_per_cta - 1) / units_per_cta;
    if (want < 1)
        want = 1;
    return (int)(want < cap ? want : cap);
}

cudaError_t write_result(stego_result *res, uint64_t msg_bytes, int status, cudaStream_t s)
{
    write_result_kernel<<<1, 1, 0, s>>>(res, msg_bytes, status);
    return cudaGetLastError();
}

} // namespace stego

// Zero at load; each slot is cleared again by the last CTA of every launch
// that used it.
static __device__ stego::StatSlot g_stat_slots[stego::kStatSlots];

namespace stego {

StatSlot *stats_slot(cudaStream_t s)
{
    if (s == cudaStreamPerThread)
        return nullptr;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
        return nullptr;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return nullptr;
    unsigned long long sid = 0;
    if (cudaStreamGetId(s, &sid) != cudaSuccess)
        return nullptr;
    // the current context's identity: 0 when it cannot be read, and then the
    // slots are not used (a stale device address would go unnoticed)
    const unsigned long long ctx = context_id();
    if (!ctx)
        return nullptr;
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_slot_ctx[dev] != ctx) {
        // first use on this device, or the device was reset since: the slot
        // array was loaded afresh (zeroed) in the new context, possibly at
        // another address, and no stream of the old context survives
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_stat_slots) != cudaSuccess || !p)
            return nullptr;
        g_slot_base[dev] = static_cast<StatSlot *>(p);
        g_slot_n[dev] = 0;
        g_slot_ctx[dev] = ctx;
    }
    for (int i = 0; i < g_slot_n[dev]; ++i)
        if (g_slot_sid[dev][i] == sid)
            return g_slot_base[dev] + i;
    if (g_slot_n[dev] == kStatSlots)
        return nullptr;
    g_slot_sid[dev][g_slot_n[dev]] = sid;
    return g_slot_base[dev] + g_slot_n[dev]++;
}

} // namespace stego

using namespace stego;

extern "C" {

int stego_version(void) { return kVersion; }

const char *stego_strerror(int status)
{
    switch (status) {
    case STEGO_OK: return "ok";
    case STEGO_E_INVAL: return "invalid argument";
    case STEGO_E_CAPACITY: return "message does not fit in the cover";
    case STEGO_E_BAD_HEADER: return "bad or missing length header";
    case STEGO_E_MSG_TOO_SMALL: return "message buffer too small";
    case STEGO_E_CUDA: return "CUDA error";
    case STEGO_E_NOMEM: return "workspace too small";
    case STEGO_E_TIMEOUT: return "device wait timed out";
    default: return "unknown status";
    }
}

int stego_capacity(uint64_t cover_bytes, const stego_geom *geom, uint32_t flags,
                   uint64_t *out_msg_bytes)
{
    if (!out_msg_bytes)
        return STEGO_E_INVAL;
    const uint32_t layout = flags & STEGO_LAYOUT_MASK;
    if (layout == STEGO_LAYOUT_STREAM1) {
        const uint32_t k = ((flags & STEGO_BITS_MASK) >> 8) + 1u;
        uint64_t carry = cover_bytes;
        if (flags & STEGO_PLANE_ONLY) {
            if (!geom_ok(geom, cover_bytes))
                return STEGO_E_INVAL;
            carry = (uint64_t)geom->width * geom->height;
        }
        uint64_t cap = carry * k / 8u;
        if (flags & STEGO_HEADER_BE32) {
            cap = cap >= 4u ? cap - 4u : 0u;
            if (cap > kMaxHeaderMsg)
                cap = kMaxHeaderMsg;
        }
        *out_msg_bytes = cap;
        return STEGO_OK;
    }
    if (layout == STEGO_LAYOUT_PAPER2) {
        if (!geom_ok(geom, cover_bytes))
            return STEGO_E_INVAL;
        *out_msg_bytes = (uint64_t)(geom->width / 4u) * geom->height;
        return STEGO_OK;
    }
    return STEGO_E_INVAL;
}

int stego_embed(const uint8_t *d_cover, uint8_t *d_stego, uint64_t cover_bytes,
                const uint8_t *d_msg, uint64_t msg_bytes, const stego_geom *geom,
                uint32_t flags, stego_result *d_result, void *stream)
{
    stego::Trace trace_("stego_embed");
    const uint32_t known = STEGO_LAYOUT_MASK | STEGO_HEADER_BE32 | STEGO_FUSE_STATS |
                           STEGO_PLANE_ONLY | STEGO_BITS_MASK;
    if (flags & ~known)
        return STEGO_E_INVAL;
    const uint32_t layout = flags & STEGO_LAYOUT_MASK;
    const bool header = (flags & STEGO_HEADER_BE32) != 0;
    const bool stats = (flags & STEGO_FUSE_STATS) != 0;
    const bool plane_only = (flags & STEGO_PLANE_ONLY) != 0;
    const uint32_t k = bits_of(flags);
    if (layout != STEGO_LAYOUT_STREAM1 && layout != STEGO_LAYOUT_PAPER2)
        return STEGO_E_INVAL;
    if (layout == STEGO_LAYOUT_PAPER2 && (header || plane_only || k != 1))
        return STEGO_E_INVAL;
    if (cover_bytes > 0 && (!d_cover || !d_stego))
        return STEGO_E_INVAL;
    if (msg_bytes > 0 && !d_msg)
        return STEGO_E_INVAL;
    if (stats && !d_result)
        return STEGO_E_INVAL;
    if (d_result && ((uintptr_t)d_result & 7u))
        return STEGO_E_INVAL;
    const bool inplace = d_stego == d_cover;
    if (!inplace && overlap(d_cover, cover_bytes, d_stego, cover_bytes))
        return STEGO_E_INVAL;
    if (overlap(d_msg, msg_bytes, d_stego, cover_bytes))
        return STEGO_E_INVAL;
    if (d_result && (overlap(d_result, sizeof(stego_result), d_stego, cover_bytes) ||
                     overlap(d_result, sizeof(stego_result), d_msg, msg_bytes) ||
                     overlap(d_result, sizeof(stego_result), d_cover, cover_bytes)))
        return STEGO_E_INVAL;
    uint64_t cap = 0;
    int st = stego_capacity(cover_bytes, geom, flags, &cap);
    if (st != STEGO_OK)
        return st;
    if (msg_bytes > cap)
        return STEGO_E_CAPACITY;
    if (layout == STEGO_LAYOUT_STREAM1 && header) {
        // the header alone needs 32 stream bits
        const uint64_t carry = plane_only ? (uint64_t)geom->width * geom->height : cover_bytes;
        if (carry * k < 32u)
            return STEGO_E_CAPACITY;
    }

    cudaStream_t s = (cudaStream_t)stream;
    const Shape sh = shape_for(STEGO_OP_EMBED, nullptr);
    // fused statistics: the stream's slot, or zeroed result fields
    StatSlot *slot = stats ? stats_slot(s) : nullptr;
    if (stats && !slot && cudaMemsetAsync(d_result, 0, 2 * sizeof(uint64_t), s) != cudaSuccess)
        return STEGO_E_CUDA;

    if (layout == STEGO_LAYOUT_STREAM1 && (k != 1 || plane_only)) {
        if (cover_bytes == 0 || (!header && msg_bytes == 0 && inplace)) {
            if (d_result)
                return cuda_status(write_result(d_result, msg_bytes, STEGO_OK, s));
            return STEGO_OK;
        }
        return cuda_status(sk_embed(d_cover, d_stego, cover_bytes, k, plane_only, geom, d_msg,
                                    msg_bytes, header, stats, d_result, sh, s, slot));
    }
    if (layout == STEGO_LAYOUT_STREAM1) {
        const uint64_t slen = msg_bytes + (header ? 4u : 0u);
        const uint64_t T = 8u * slen;
        const uint64_t n = inplace ? T : cover_bytes;
        if (n == 0) {
            if (d_result)
                return cuda_status(write_result(d_result, msg_bytes, STEGO_OK, s));
            return STEGO_OK;
        }
        return cuda_status(s1_embed(d_cover, d_stego, n, T, d_msg, slen, header,
                                    (uint32_t)(8u * msg_bytes), stats, d_result, msg_bytes, sh, s,
                                    slot));
    }
    // PAPER2 out of place: one fused pass when the layout allows it
    if (!inplace && cover_bytes > 0 && p2_fused_ok(d_cover, d_stego, *geom))
        return cuda_status(p2_embed_fused(d_cover, d_stego, *geom, d_msg, msg_bytes, stats,
                                          d_result, sh, s, slot));
    // otherwise copy the cover (out of place), then write the 4N carrying bytes
    if (!inplace && cover_bytes > 0) {
        cudaError_t e = s1_embed(d_cover, d_stego, cover_bytes, 0, nullptr, 0, false, 0, false,
                                 msg_bytes == 0 ? d_result : nullptr, 0, sh, s);
        if (e != cudaSuccess)
            return STEGO_E_CUDA;
        if (msg_bytes == 0)
            return STEGO_OK;
    }
    if (msg_bytes == 0) {
        if (d_result)
            return cuda_status(write_result(d_result, 0, STEGO_OK, s));
        return STEGO_OK;
    }
    return cuda_status(p2_embed(d_cover, d_stego, *geom, d_msg, msg_bytes, stats, d_result, sh, s,
                                slot));
}

} // extern "C"

namespace {

// stego_extract and stego_extract_ballot: validation and dispatch; with
// `ballot` the one-bit stream layout's kernel packs the message by ballots.
int extract_impl(const uint8_t *d_stego, uint64_t cover_bytes, uint8_t *d_msg,
                 uint64_t msg_cap, uint64_t msg_len, const stego_geom *geom, uint32_t flags,
                 stego_result *d_result, void *stream, bool ballot)
{
    const uint32_t known = STEGO_LAYOUT_MASK | STEGO_HEADER_BE32 | STEGO_PLANE_ONLY |
                           STEGO_BITS_MASK;
    if (flags & ~known)
        return STEGO_E_INVAL;
    const uint32_t layout = flags & STEGO_LAYOUT_MASK;
    const bool header = (flags & STEGO_HEADER_BE32) != 0;
    const bool plane_only = (flags & STEGO_PLANE_ONLY) != 0;
    const uint32_t k = bits_of(flags);
    if (layout != STEGO_LAYOUT_STREAM1 && layout != STEGO_LAYOUT_PAPER2)
        return STEGO_E_INVAL;
    if (ballot && (layout != STEGO_LAYOUT_STREAM1 || plane_only || k != 1))
        return STEGO_E_INVAL;
    if (layout == STEGO_LAYOUT_PAPER2 && (header || plane_only || k != 1))
        return STEGO_E_INVAL;
    if (plane_only && !geom_ok(geom, cover_bytes))
        return STEGO_E_INVAL;
    if (cover_bytes > 0 && !d_stego)
        return STEGO_E_INVAL;
    if (header && !d_result)
        return STEGO_E_INVAL;
    if (d_result && ((uintptr_t)d_result & 7u))
        return STEGO_E_INVAL;
    if (msg_cap > 0 && !d_msg)
        return STEGO_E_INVAL;
    if (overlap(d_msg, msg_cap, d_stego, cover_bytes))
        return STEGO_E_INVAL;
    if (d_result && (overlap(d_result, sizeof(stego_result), d_msg, msg_cap) ||
                     overlap(d_result, sizeof(stego_result), d_stego, cover_bytes)))
        return STEGO_E_INVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const Shape sh = shape_for(STEGO_OP_EXTRACT, nullptr);

    const bool variant = layout == STEGO_LAYOUT_STREAM1 && (k != 1 || plane_only);
    if (layout == STEGO_LAYOUT_STREAM1 && header) {
        // length and status come from the device
        if (variant)
            return cuda_status(sk_extract(d_stego, cover_bytes, k, plane_only, geom, d_msg,
                                          msg_cap, 0, true, d_result, sh, s));
        if (ballot)
            return cuda_status(s1_extract_ballot(d_stego, cover_bytes, d_msg, msg_cap, 0, true,
                                                 d_result, sh, s));
        return cuda_status(s1_extract(d_stego, cover_bytes, d_msg, msg_cap, 0, true, d_result, sh, s));
    }
    uint64_t cap = 0;
    int st = stego_capacity(cover_bytes, geom, flags, &cap);
    if (st != STEGO_OK)
        return st;
    if (msg_len > cap)
        return STEGO_E_CAPACITY;
    if (msg_len > msg_cap)
        return STEGO_E_MSG_TOO_SMALL;
    if (msg_len == 0) {
        if (d_result)
            return cuda_status(write_result(d_result, 0, STEGO_OK, s));
        return STEGO_OK;
    }
    if (variant)
        return cuda_status(sk_extract(d_stego, cover_bytes, k, plane_only, geom, d_msg, msg_cap,
                                      msg_len, false, d_result, sh, s));
    if (layout == STEGO_LAYOUT_STREAM1 && ballot)
        return cuda_status(s1_extract_ballot(d_stego, cover_bytes, d_msg, msg_cap, msg_len, false,
                                             d_result, sh, s));
    if (layout == STEGO_LAYOUT_STREAM1)
        return cuda_status(s1_extract(d_stego, cover_bytes, d_msg, msg_cap, msg_len, false, d_result, sh, s));
    return cuda_status(p2_extract(d_stego, *geom, d_msg, msg_len, d_result, sh, s));
}

} // namespace

extern "C" {

int stego_extract(const uint8_t *d_stego, uint64_t cover_bytes, uint8_t *d_msg,
                  uint64_t msg_cap, uint64_t msg_len, const stego_geom *geom, uint32_t flags,
                  stego_result *d_result, void *stream)
{
    stego::Trace trace_("stego_extract");
    return extract_impl(d_stego, cover_bytes, d_msg, msg_cap, msg_len, geom, flags, d_result,
                        stream, false);
}

int stego_extract_ballot(const uint8_t *d_stego, uint64_t cover_bytes, uint8_t *d_msg,
                         uint64_t msg_cap, uint64_t msg_len, const stego_geom *geom,
                         uint32_t flags, stego_result *d_result, void *stream)
{
    stego::Trace trace_("stego_extract_ballot");
    return extract_impl(d_stego, cover_bytes, d_msg, msg_cap, msg_len, geom, flags, d_result,
                        stream, true);
}

int stego_changed_bytes(const uint8_t *d_a, const uint8_t *d_b, uint64_t n, uint64_t *d_out2,
                        void *stream)
{
    stego::Trace trace_("stego_changed_bytes");
    if (!d_out2 || ((uintptr_t)d_out2 & 7u))
        return STEGO_E_INVAL;
    if (n > 0 && (!d_a || !d_b))
        return STEGO_E_INVAL;
    if (overlap(d_out2, 2 * sizeof(uint64_t), d_a, n) || overlap(d_out2, 2 * sizeof(uint64_t), d_b, n))
        return STEGO_E_INVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemsetAsync(d_out2, 0, 2 * sizeof(uint64_t), s) != cudaSuccess)
        return STEGO_E_CUDA;
    if (n == 0)
        return STEGO_OK;
    const Shape sh = shape_for(STEGO_OP_CHANGED, nullptr);
    return cuda_status(changed_bytes(d_a, d_b, n, reinterpret_cast<unsigned long long *>(d_out2), sh, s));
}

int stego_pointer_kind(const void *p, int *kind, int *device_accessible)
{
    if (!kind || !device_accessible)
        return STEGO_E_INVAL;
    *kind = STEGO_MEM_PAGEABLE;
    *device_accessible = 0;
    cudaPointerAttributes at;
    std::memset(&at, 0, sizeof(at));
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return STEGO_E_CUDA;
    }
    switch (at.type) {
    case cudaMemoryTypeDevice:
        *kind = STEGO_MEM_DEVICE;
        *device_accessible = 1;
        break;
    case cudaMemoryTypeManaged:
        *kind = STEGO_MEM_MANAGED;
        *device_accessible = 1;
        break;
    case cudaMemoryTypeHost:
        *kind = STEGO_MEM_PINNED;
        *device_accessible = at.devicePointer == p ? 1 : 0;
        break;
    default: {
        int dev = 0, pageable = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, dev) != cudaSuccess)
            pageable = 0;
        *kind = STEGO_MEM_PAGEABLE;
        *device_accessible = pageable ? 1 : 0;
        break;
    }
    }
    return STEGO_OK;
}

int stego_set_tune(int op, const stego_tune *t)
{
    if (op < 0 || op >= STEGO_OP_COUNT || !t || !valid_tune_field_ranges(*t))
        return STEGO_E_INVAL;
    std::lock_guard<std::mutex> lk(g_mu);
    Shape &s = g_shape[op];
    if (t->threads)
        s.threads = (int)t->threads;
    if (t->vec_per_thread)
        s.vec = (int)t->vec_per_thread;
    s.ctas_per_sm = (int)t->ctas_per_sm; // 0 restores "occupancy maximum"
    // single-cover calls: 0 selects the register kernels, so it is installed too
    if (t->tile_bytes || op == STEGO_OP_EMBED || op == STEGO_OP_EXTRACT)
        s.tile_bytes = t->tile_bytes;
    return STEGO_OK;
}

int stego_get_tune(int op, stego_tune *out)
{
    if (op < 0 || op >= STEGO_OP_COUNT || !out)
        return STEGO_E_INVAL;
    std::lock_guard<std::mutex> lk(g_mu);
    const Shape &s = g_shape[op];
    out->threads = (uint32_t)s.threads;
    out->vec_per_thread = (uint32_t)s.vec;
    out->ctas_per_sm = (uint32_t)s.ctas_per_sm;
    out->tile_bytes = s.tile_bytes;
    return STEGO_OK;
}

} // extern "C"

static_assert(sizeof(stego_desc) == 72, "stego_desc layout");
static_assert(sizeof(stego_result) == 32, "stego_result layout");
static_assert(sizeof(stego_geom) == 16, "stego_geom layout");
static_assert(sizeof(stego_tune) == 16, "stego_tune layout");
static_assert(sizeof(stego::StatSlot) == 32, "statistics slot layout");
static_assert(sizeof(stego_request) == 80, "stego_request layout");
static_assert(sizeof(stego_completion) == 64, "stego_completion layout");
static_assert(sizeof(stego_server_config) == 48, "stego_server_config layout");
