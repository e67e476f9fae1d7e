// pipeline.cu -- batched embed / extract of covers that live in host memory,
// with the copies in both directions overlapped with the kernels.
//
// The paper's gateway (Section V) allocates device memory, copies the image
// row in, runs the kernel and copies the result out, once per row and
// frame.  Here a batch of host-resident jobs is cut into chunks that fit one
// device staging slot; chunk k uses slot k mod S and runs as three
// stream-ordered stages on three streams:
//   copy in    descriptors, covers and messages, host -> slot;
//   compute    one batched embed in place on the slot (and, for jobs that
//              ask for it, one batched extract of the new stegos: the
//              read-back), or one batched extract;
//   copy out   stegos, read-back messages and results, slot -> host.
// Events chain the stages of a chunk and keep a slot's next copy-in behind
// its last copy-out, so with two or more slots chunk k+1's copy-in, chunk
// k's kernels and chunk k-1's copy-out run at the same time: both link
// directions and the SMs are busy together.
//
// Extraction writes each message straight into the caller's host buffer
// (the batched kernel stores through the mapped pinned pointer), so only
// the extracted bytes are written, as in the device-resident calls.
//
// In the automatic mode only jobs that reuse data on the device are staged
// (an embed whose stego is read back: the extraction reads the slot, not
// the host).  Every other job is zero copy: its descriptor points at the
// host buffers and the batched kernels read and write them over the
// CPU-GPU link, the cover and stego traffic of all such jobs overlapping in
// one launch per chunk, and an extraction reading only the stego's carrying
// bytes (measured on the 4096-cover batch: 165 against 130 cover GB/s
// staged for the embed, 383 against 181 for the extraction).  The staged
// mode stages every job.
//
// Device memory: one caller-owned arena (stego_pipeline_arena_bytes) holds
// every slot's descriptors, results, batched workspace and data area; the
// pipeline allocates no device memory.  Its pinned host staging for
// descriptors and results is allocated once, at creation.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include <cuda.h>

#include "internal.cuh"

namespace {

constexpr uint32_t kMaxSlots = 8;
constexpr uint32_t kMaxDescs = 8192;
// bytes past each slot's data area that a vector load at the end of the
// last cover may touch (the kernels never read this far, the pad only keeps
// any such read inside the arena)
constexpr uint64_t kSlotPad = 4096;

uint64_t up256(uint64_t x) { return (x + 255u) & ~255ull; }

struct Layout {
    uint64_t desc, desc_rb, res, res_rb, ws, data, per_slot;
};

Layout layout_of(const stego_pipeline_config &c)
{
    Layout L;
    const uint64_t m = c.max_descs;
    uint64_t o = 0;
    L.desc = o;
    o += up256(sizeof(stego_desc) * m);
    L.desc_rb = o;
    o += up256(sizeof(stego_desc) * m);
    L.res = o;
    o += up256(sizeof(stego_result) * m);
    L.res_rb = o;
    o += up256(sizeof(stego_result) * m);
    L.ws = o;
    o += up256(stego_batched_workspace_bytes(c.max_descs));
    L.data = o;
    o += up256(c.slot_bytes) + kSlotPad;
    L.per_slot = up256(o);
    return L;
}

bool config_ok(const stego_pipeline_config *c)
{
    return c && c->slots >= 1 && c->slots <= kMaxSlots && c->max_descs >= 1 &&
           c->max_descs <= kMaxDescs && c->slot_bytes >= 4096 &&
           (c->mode == STEGO_PIPE_AUTO || c->mode == STEGO_PIPE_STAGED) && c->reserved == 0 &&
           stego::tune_ok(&c->tune_embed) && stego::tune_ok(&c->tune_extract);
}

bool overlap(const void *p, uint64_t np, const void *q, uint64_t nq)
{
    if (np == 0 || nq == 0 || p == nullptr || q == nullptr)
        return false;
    const uintptr_t a = (uintptr_t)p, b = (uintptr_t)q;
    return a < b + nq && b < a + np;
}

bool geom_ok(const stego_geom &g, uint64_t cover_bytes)
{
    return g.channels > 0 && g.plane < g.channels &&
           (uint64_t)g.width * g.height * g.channels == cover_bytes;
}

// The embed's argument checks (the batched call's per-cover checks, made on
// the host so that a refused job is never staged or copied back).
int embed_job_status(const stego_host_job &j)
{
    const uint32_t layout = j.flags & STEGO_LAYOUT_MASK;
    const bool header = (j.flags & STEGO_HEADER_BE32) != 0;
    if (j.flags & ~(STEGO_LAYOUT_MASK | STEGO_HEADER_BE32 | STEGO_FUSE_STATS))
        return STEGO_E_INVAL;
    if (layout != STEGO_LAYOUT_STREAM1 && layout != STEGO_LAYOUT_PAPER2)
        return STEGO_E_INVAL;
    if (j.cover_bytes > 0 && (!j.cover || !j.stego))
        return STEGO_E_INVAL;
    if (j.msg_bytes > 0 && !j.msg)
        return STEGO_E_INVAL;
    if (j.stego != j.cover && overlap(j.cover, j.cover_bytes, j.stego, j.cover_bytes))
        return STEGO_E_INVAL;
    if (overlap(j.msg, j.msg_bytes, j.stego, j.cover_bytes))
        return STEGO_E_INVAL;
    if (j.readback && (overlap(j.readback, j.msg_bytes, j.stego, j.cover_bytes) ||
                       overlap(j.readback, j.msg_bytes, j.cover, j.cover_bytes) ||
                       overlap(j.readback, j.msg_bytes, j.msg, j.msg_bytes)))
        return STEGO_E_INVAL;
    if (layout == STEGO_LAYOUT_PAPER2) {
        if (header || !geom_ok(j.geom, j.cover_bytes))
            return STEGO_E_INVAL;
        if (j.msg_bytes > (uint64_t)(j.geom.width / 4u) * j.geom.height)
            return STEGO_E_CAPACITY;
        return STEGO_OK;
    }
    uint64_t cap = j.cover_bytes / 8u;
    if (header) {
        cap = cap >= 4u ? cap - 4u : 0u;
        if (cap > 0x1FFFFFFFull)
            cap = 0x1FFFFFFFull;
    }
    if (j.msg_bytes > cap || (header && j.cover_bytes < 32))
        return STEGO_E_CAPACITY;
    return STEGO_OK;
}

// Cover bytes an embed can change: with the stego in place in host memory
// only this prefix is copied in and back.
uint64_t embed_prefix(const stego_host_job &j)
{
    if ((j.flags & STEGO_LAYOUT_MASK) == STEGO_LAYOUT_PAPER2) {
        const uint64_t per_row = j.geom.width / 4u;
        if (j.msg_bytes == 0 || per_row == 0)
            return 0;
        const uint64_t rows = (j.msg_bytes + per_row - 1) / per_row;
        return rows * j.geom.width * j.geom.channels;
    }
    const uint64_t slen = j.msg_bytes + ((j.flags & STEGO_HEADER_BE32) ? 4u : 0u);
    return std::min<uint64_t>(j.cover_bytes, 8u * slen);
}

// Largest hole between two host buffers of one allocation that are still
// copied in as one range (the hole's bytes are copied too).
constexpr uint64_t kMergeGap = 64u << 10;

struct Staged {
    uint32_t job;
    uint64_t in_bytes;  // cover bytes copied in (the slot holds all cover_bytes)
    uint64_t out_bytes; // embed: stego bytes copied back
    bool zero_copy;     // the kernels use the job's host buffers directly
    uint64_t cover_off; // offsets in the slot's data area (set at launch)
    uint64_t msg_off;
    uint64_t rb_off;
};

// Allocation that contains a host pointer, as the driver reports it (pinned
// host memory lives in the unified address space); false when unknown.
using PtrAttrFn = CUresult(CUDAAPI *)(void *, CUpointer_attribute, CUdeviceptr);
std::once_flag g_attr_once;
PtrAttrFn g_ptr_attr = nullptr;

bool alloc_range(const void *ptr, uintptr_t &start, uintptr_t &size)
{
    std::call_once(g_attr_once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuPointerGetAttribute", &f, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ptr_attr = reinterpret_cast<PtrAttrFn>(f);
    });
    if (!g_ptr_attr)
        return false;
    CUdeviceptr st = 0;
    size_t sz = 0;
    if (g_ptr_attr(&st, CU_POINTER_ATTRIBUTE_RANGE_START_ADDR, (CUdeviceptr)(uintptr_t)ptr) !=
            CUDA_SUCCESS ||
        g_ptr_attr(&sz, CU_POINTER_ATTRIBUTE_RANGE_SIZE, (CUdeviceptr)(uintptr_t)ptr) !=
            CUDA_SUCCESS) {
        cudaGetLastError();
        return false;
    }
    start = (uintptr_t)st;
    size = (uintptr_t)sz;
    return start <= (uintptr_t)ptr && (uintptr_t)ptr < start + size;
}

// Places host ranges in a slot's data area from `cursor` on, one copy per
// run: consecutive ranges that ascend inside one allocation with holes of at
// most kMergeGap, whose offsets from the run's first range are multiples of
// `mod`, keep their relative offsets (the run starts on a 16-byte boundary,
// so with mod = 16 every range of it is 16-byte aligned on the device).
struct RunPlacer {
    uint64_t cursor;
    uint64_t mod;
    const uint8_t *run_host = nullptr; // first byte of the open run
    const uint8_t *run_end = nullptr;
    uint64_t run_dev = 0;
    uintptr_t a_start = 0, a_size = 0; // allocation of the open run
    bool a_known = false;

    // Device offset of a range of `len` bytes at ptr of which the first
    // `copy_len` are copied in; `copy` is told to copy a finished run (host,
    // device offset, bytes).  A range copied in part is placed alone.
    template <typename Copy>
    uint64_t place(const uint8_t *ptr, uint64_t len, uint64_t copy_len, Copy &&copy)
    {
        if (len == 0)
            return cursor;
        if (copy_len < len) {
            close(copy);
            const uint64_t dev = up256(cursor);
            if (copy_len)
                copy(ptr, dev, copy_len);
            cursor = dev + len;
            return dev;
        }
        if (run_host && ptr >= run_end && (uint64_t)(ptr - run_end) <= kMergeGap &&
            (uint64_t)(ptr - run_host) % mod == 0 && a_known &&
            (uintptr_t)ptr >= a_start && (uintptr_t)ptr + len <= a_start + a_size) {
            run_end = ptr + len;
            return run_dev + (uint64_t)(ptr - run_host);
        }
        close(copy);
        run_host = ptr;
        run_end = ptr + len;
        run_dev = up256(cursor) + ((uintptr_t)ptr & 255u & ~(uintptr_t)15u);
        a_known = alloc_range(ptr, a_start, a_size) && (uintptr_t)ptr + len <= a_start + a_size;
        return run_dev;
    }

    template <typename Copy> void close(Copy &&copy)
    {
        if (!run_host)
            return;
        copy(run_host, run_dev, (uint64_t)(run_end - run_host));
        cursor = run_dev + (uint64_t)(run_end - run_host);
        run_host = run_end = nullptr;
    }
};

// Upper bound of the slot bytes a range adds after `prev_end` (its run
// either grows by the hole and the range, or a new run starts on the next
// 16-byte boundary past a 256-byte boundary).
uint64_t placement_bound(const uint8_t *prev_end, const uint8_t *ptr, uint64_t len)
{
    uint64_t hole = 0;
    if (prev_end && ptr >= prev_end && (uint64_t)(ptr - prev_end) <= kMergeGap)
        hole = (uint64_t)(ptr - prev_end);
    return len + hole + 512u;
}

struct SlotState {
    cudaEvent_t in_done = nullptr, comp_done = nullptr, out_done = nullptr;
    stego_desc *h_desc = nullptr, *h_desc_rb = nullptr;
    stego_result *h_res = nullptr, *h_res_rb = nullptr;
    std::vector<Staged> jobs; // the chunk in flight on this slot
    bool busy = false;
    bool readback = false;
    int launch_status = STEGO_OK;
};

} // namespace

struct stego_pipeline {
    stego_pipeline_config cfg;
    Layout L;
    char *arena = nullptr;
    cudaStream_t s_in = nullptr, s_comp = nullptr, s_out = nullptr;
    SlotState slot[kMaxSlots];
    int device = 0;
    int pageable_access = 0; // the device's kernels may touch pageable host memory
};

namespace {

// A kernel reads or writes through the caller's pointer (an extraction's
// message; every buffer of a zero-copy job): it must be one the device may
// dereference.
bool kernel_can_write(const stego_pipeline *p, const void *ptr)
{
    if (p->pageable_access || !ptr)
        return true;
    cudaPointerAttributes at;
    std::memset(&at, 0, sizeof(at));
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged)
        return true;
    return at.type == cudaMemoryTypeHost && at.devicePointer == ptr;
}

char *slot_base(stego_pipeline *p, uint32_t j) { return p->arena + (uint64_t)j * p->L.per_slot; }

// Results of the chunk last run on slot j into the caller's arrays.
int harvest(stego_pipeline *p, uint32_t j, const stego_host_job *jobs, stego_result *results,
            stego_result *rb_results)
{
    SlotState &sl = p->slot[j];
    if (!sl.busy)
        return STEGO_OK;
    sl.busy = false;
    if (cudaEventSynchronize(sl.out_done) != cudaSuccess)
        return STEGO_E_CUDA;
    for (size_t i = 0; i < sl.jobs.size(); ++i) {
        const uint32_t k = sl.jobs[i].job;
        results[k] = sl.h_res[i];
        if (rb_results) {
            if (jobs[k].readback)
                rb_results[k] = sl.h_res_rb[i];
            else
                std::memset(&rb_results[k], 0, sizeof(stego_result));
        }
    }
    sl.jobs.clear();
    return sl.launch_status;
}

cudaError_t h2d(void *dst, const void *src, uint64_t n, cudaStream_t s)
{
    return n ? cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, s) : cudaSuccess;
}

cudaError_t d2h(void *dst, const void *src, uint64_t n, cudaStream_t s)
{
    return n ? cudaMemcpyAsync(dst, src, n, cudaMemcpyDeviceToHost, s) : cudaSuccess;
}

// Copy-in, kernels and copy-out of one chunk on slot j.
int launch_chunk(stego_pipeline *p, uint32_t j, const stego_host_job *jobs, bool embed,
                 uint32_t flags)
{
    stego::Trace trace_("stego_pipeline chunk");
    SlotState &sl = p->slot[j];
    char *base = slot_base(p, j);
    uint8_t *data = reinterpret_cast<uint8_t *>(base + p->L.data);
    stego_desc *d_desc = reinterpret_cast<stego_desc *>(base + p->L.desc);
    stego_desc *d_desc_rb = reinterpret_cast<stego_desc *>(base + p->L.desc_rb);
    stego_result *d_res = reinterpret_cast<stego_result *>(base + p->L.res);
    stego_result *d_res_rb = reinterpret_cast<stego_result *>(base + p->L.res_rb);
    void *d_ws = base + p->L.ws;
    const uint64_t ws_bytes = stego_batched_workspace_bytes(p->cfg.max_descs);
    const uint32_t n = (uint32_t)sl.jobs.size();
    // copy in, once the slot's previous chunk has been copied out; the
    // covers' and messages' runs are copied as they are closed
    cudaError_t e = cudaStreamWaitEvent(p->s_in, sl.out_done, 0);
    auto copy_in = [&](const uint8_t *host, uint64_t dev_off, uint64_t bytes) {
        if (e == cudaSuccess)
            e = h2d(data + dev_off, host, bytes, p->s_in);
    };
    RunPlacer covers{0, 16};
    for (uint32_t i = 0; i < n; ++i) {
        Staged &g = sl.jobs[i];
        if (!g.zero_copy)
            g.cover_off = covers.place(jobs[g.job].cover, jobs[g.job].cover_bytes, g.in_bytes,
                                       copy_in);
    }
    covers.close(copy_in);
    RunPlacer msgs{covers.cursor, 2};
    for (uint32_t i = 0; i < n && embed; ++i) {
        Staged &g = sl.jobs[i];
        if (!g.zero_copy)
            g.msg_off = msgs.place(jobs[g.job].msg, jobs[g.job].msg_bytes,
                                   jobs[g.job].msg_bytes, copy_in);
    }
    msgs.close(copy_in);
    uint64_t cursor = up256(msgs.cursor);
    sl.readback = false;
    for (uint32_t i = 0; i < n; ++i) {
        Staged &g = sl.jobs[i];
        const stego_host_job &J = jobs[g.job];
        g.rb_off = cursor;
        if (embed && J.readback)
            cursor += up256(J.msg_bytes);
        stego_desc &D = sl.h_desc[i];
        std::memset(&D, 0, sizeof(D));
        D.cover = g.zero_copy ? J.cover : data + g.cover_off;
        D.cover_bytes = J.cover_bytes;
        D.flags = J.flags & (STEGO_LAYOUT_MASK | STEGO_HEADER_BE32);
        D.geom = J.geom;
        if (embed) {
            // zero copy: the host buffers themselves; staged: in place on the slot
            D.stego = g.zero_copy ? J.stego : data + g.cover_off;
            D.msg = g.zero_copy ? J.msg : data + g.msg_off;
            D.msg_bytes = J.msg_bytes;
            // the read-back extraction (an empty raw extraction for jobs
            // that do not ask for one)
            stego_desc &R = sl.h_desc_rb[i];
            std::memset(&R, 0, sizeof(R));
            if (J.readback) {
                sl.readback = true;
                R.cover = data + g.cover_off;
                R.cover_bytes = J.cover_bytes;
                R.flags = D.flags;
                R.geom = J.geom;
                R.msg = data + g.rb_off;
                R.msg_bytes = J.msg_bytes;
                R.msg_len = J.msg_bytes;
            }
        } else {
            D.msg = J.msg; // written by the kernel straight into host memory
            D.msg_bytes = J.msg_bytes;
            D.msg_len = J.msg_len;
        }
    }
    if (e == cudaSuccess)
        e = h2d(d_desc, sl.h_desc, sizeof(stego_desc) * n, p->s_in);
    if (e == cudaSuccess && sl.readback)
        e = h2d(d_desc_rb, sl.h_desc_rb, sizeof(stego_desc) * n, p->s_in);
    if (e == cudaSuccess)
        e = cudaEventRecord(sl.in_done, p->s_in);
    if (e == cudaSuccess)
        e = cudaStreamWaitEvent(p->s_comp, sl.in_done, 0);
    if (e != cudaSuccess)
        return STEGO_E_CUDA;
    // kernels
    int st;
    if (embed) {
        st = stego_embed_batched(d_desc, n, d_res, flags & STEGO_FUSE_STATS, &p->cfg.tune_embed,
                                 d_ws, ws_bytes, p->s_comp);
        if (st == STEGO_OK && sl.readback)
            st = stego_extract_batched(d_desc_rb, n, d_res_rb, 0, &p->cfg.tune_extract, d_ws,
                                       ws_bytes, p->s_comp);
    } else {
        st = stego_extract_batched(d_desc, n, d_res, 0, &p->cfg.tune_extract, d_ws, ws_bytes,
                                   p->s_comp);
    }
    if (st != STEGO_OK)
        return st;
    e = cudaEventRecord(sl.comp_done, p->s_comp);
    if (e == cudaSuccess)
        e = cudaStreamWaitEvent(p->s_out, sl.comp_done, 0);
    // copy out
    for (uint32_t i = 0; i < n && e == cudaSuccess && embed; ++i) {
        const Staged &g = sl.jobs[i];
        const stego_host_job &J = jobs[g.job];
        e = d2h(J.stego, data + g.cover_off, g.out_bytes, p->s_out);
        if (e == cudaSuccess && J.readback)
            e = d2h(J.readback, data + g.rb_off, J.msg_bytes, p->s_out);
    }
    if (e == cudaSuccess)
        e = d2h(sl.h_res, d_res, sizeof(stego_result) * n, p->s_out);
    if (e == cudaSuccess && sl.readback)
        e = d2h(sl.h_res_rb, d_res_rb, sizeof(stego_result) * n, p->s_out);
    if (e == cudaSuccess)
        e = cudaEventRecord(sl.out_done, p->s_out);
    return e == cudaSuccess ? STEGO_OK : STEGO_E_CUDA;
}

int run(stego_pipeline *p, const stego_host_job *jobs, uint32_t n, stego_result *results,
        stego_result *rb_results, uint32_t flags, bool embed)
{
    if (!p)
        return STEGO_E_INVAL;
    if (embed ? (flags & ~(uint32_t)STEGO_FUSE_STATS) != 0 : flags != 0)
        return STEGO_E_INVAL;
    if (n == 0)
        return STEGO_OK;
    if (!jobs || !results)
        return STEGO_E_INVAL;
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess)
        return STEGO_E_CUDA;
    if (cur != p->device && cudaSetDevice(p->device) != cudaSuccess)
        return STEGO_E_CUDA;
    const uint64_t cap = p->cfg.slot_bytes;
    int status = STEGO_OK;
    uint32_t next_slot = 0;
    std::vector<Staged> chunk;
    // slot bytes the chunk may use: 256 for the read-back area's alignment,
    // then each job's placement bound
    uint64_t used = 256;
    const uint8_t *prev_cover = nullptr, *prev_msg = nullptr; // ends of the chunk's last ranges

    auto flush = [&]() -> int {
        if (chunk.empty())
            return STEGO_OK;
        const uint32_t j = next_slot;
        next_slot = (next_slot + 1) % p->cfg.slots;
        int st = harvest(p, j, jobs, results, rb_results);
        if (st != STEGO_OK)
            return st;
        SlotState &sl = p->slot[j];
        sl.jobs.swap(chunk);
        chunk.clear();
        used = 256;
        prev_cover = prev_msg = nullptr;
        sl.busy = true;
        sl.launch_status = launch_chunk(p, j, jobs, embed, flags);
        return sl.launch_status;
    };

    for (uint32_t k = 0; k < n && status == STEGO_OK; ++k) {
        const stego_host_job &J = jobs[k];
        int st = STEGO_OK;
        Staged g;
        std::memset(&g, 0, sizeof(g));
        g.job = k;
        if (embed) {
            st = embed_job_status(J);
            // without a read-back nothing is reused on the device: in the
            // automatic mode the kernel reads and writes the host buffers
            g.zero_copy = p->cfg.mode == STEGO_PIPE_AUTO && !J.readback &&
                          kernel_can_write(p, J.cover) && kernel_can_write(p, J.stego) &&
                          kernel_can_write(p, J.msg);
            if (g.zero_copy)
                g.in_bytes = g.out_bytes = 0;
            else if (J.stego == J.cover) // in place in host memory: the bytes that can change
                g.in_bytes = g.out_bytes = embed_prefix(J);
            else
                g.in_bytes = g.out_bytes = J.cover_bytes;
        } else {
            // the header's checks run on the device; the cover is copied whole
            if (J.cover_bytes > 0 && !J.cover)
                st = STEGO_E_INVAL;
            else if (J.msg_bytes > 0 && !J.msg)
                st = STEGO_E_INVAL;
            else if (overlap(J.msg, J.msg_bytes, J.cover, J.cover_bytes))
                st = STEGO_E_INVAL;
            else if (J.msg_bytes > 0 && !kernel_can_write(p, J.msg))
                st = STEGO_E_INVAL;
            // the automatic mode reads the stego where it is: only the
            // carrying bytes cross the link
            g.zero_copy = p->cfg.mode == STEGO_PIPE_AUTO && kernel_can_write(p, J.cover);
            g.in_bytes = g.zero_copy ? 0 : J.cover_bytes;
        }
        // slot bytes this job may add, alone and behind the chunk's last job
        const uint64_t rb = embed && J.readback ? up256(J.msg_bytes) : 0;
        const uint64_t alone =
            g.zero_copy ? 256u
                        : 256u + J.cover_bytes + 512u + (embed ? J.msg_bytes + 512u : 0) + rb;
        if (st == STEGO_OK && alone > cap)
            st = STEGO_E_NOMEM; // larger than a whole slot
        if (st != STEGO_OK) {
            std::memset(&results[k], 0, sizeof(stego_result));
            results[k].status = st;
            if (rb_results) {
                std::memset(&rb_results[k], 0, sizeof(stego_result));
                rb_results[k].status = st;
            }
            continue;
        }
        const bool part = g.in_bytes < J.cover_bytes; // placed alone
        uint64_t need =
            g.zero_copy ? 0
                        : placement_bound(part ? nullptr : prev_cover, J.cover, J.cover_bytes) +
                              rb + (embed ? placement_bound(prev_msg, J.msg, J.msg_bytes) : 0);
        if (chunk.size() == p->cfg.max_descs || used + need > cap) {
            status = flush();
            if (status != STEGO_OK)
                break;
            need = alone - 256u;
        }
        used += need;
        if (!g.zero_copy) {
            if (part)
                prev_cover = nullptr;
            else if (J.cover_bytes)
                prev_cover = J.cover + J.cover_bytes;
            if (embed && J.msg_bytes)
                prev_msg = J.msg + J.msg_bytes;
        }
        chunk.push_back(g);
    }
    if (status == STEGO_OK)
        status = flush();
    // every chunk in flight, in launch order
    for (uint32_t i = 0; i < p->cfg.slots; ++i) {
        const int st = harvest(p, (next_slot + i) % p->cfg.slots, jobs, results, rb_results);
        if (status == STEGO_OK)
            status = st;
    }
    if (cur != p->device)
        cudaSetDevice(cur);
    return status;
}

void release(stego_pipeline *p)
{
    for (uint32_t j = 0; j < kMaxSlots; ++j) {
        SlotState &sl = p->slot[j];
        if (sl.in_done)
            cudaEventDestroy(sl.in_done);
        if (sl.comp_done)
            cudaEventDestroy(sl.comp_done);
        if (sl.out_done)
            cudaEventDestroy(sl.out_done);
        cudaFreeHost(sl.h_desc);
        cudaFreeHost(sl.h_desc_rb);
        cudaFreeHost(sl.h_res);
        cudaFreeHost(sl.h_res_rb);
    }
    if (p->s_in)
        cudaStreamDestroy(p->s_in);
    if (p->s_comp)
        cudaStreamDestroy(p->s_comp);
    if (p->s_out)
        cudaStreamDestroy(p->s_out);
    delete p;
}

} // namespace

extern "C" {

uint64_t stego_pipeline_arena_bytes(const stego_pipeline_config *cfg)
{
    if (!config_ok(cfg))
        return 0;
    return layout_of(*cfg).per_slot * cfg->slots;
}

int stego_pipeline_create(const stego_pipeline_config *cfg, void *d_arena, uint64_t arena_bytes,
                          stego_pipeline **out)
{
    if (!out)
        return STEGO_E_INVAL;
    *out = nullptr;
    if (!config_ok(cfg) || !d_arena || ((uintptr_t)d_arena & 255u))
        return STEGO_E_INVAL;
    if (arena_bytes < stego_pipeline_arena_bytes(cfg))
        return STEGO_E_NOMEM;
    stego_pipeline *p = new stego_pipeline;
    p->cfg = *cfg;
    p->L = layout_of(*cfg);
    p->arena = static_cast<char *>(d_arena);
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        delete p;
        return STEGO_E_CUDA;
    }
    if (cudaDeviceGetAttribute(&p->pageable_access, cudaDevAttrPageableMemoryAccess,
                               p->device) != cudaSuccess)
        p->pageable_access = 0;
    bool ok = cudaStreamCreateWithFlags(&p->s_in, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&p->s_comp, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&p->s_out, cudaStreamNonBlocking) == cudaSuccess;
    const size_t dsz = sizeof(stego_desc) * cfg->max_descs;
    const size_t rsz = sizeof(stego_result) * cfg->max_descs;
    for (uint32_t j = 0; ok && j < cfg->slots; ++j) {
        SlotState &sl = p->slot[j];
        ok = cudaEventCreateWithFlags(&sl.in_done, cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&sl.comp_done, cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&sl.out_done, cudaEventDisableTiming) == cudaSuccess &&
             cudaHostAlloc((void **)&sl.h_desc, dsz, cudaHostAllocDefault) == cudaSuccess &&
             cudaHostAlloc((void **)&sl.h_desc_rb, dsz, cudaHostAllocDefault) == cudaSuccess &&
             cudaHostAlloc((void **)&sl.h_res, rsz, cudaHostAllocDefault) == cudaSuccess &&
             cudaHostAlloc((void **)&sl.h_res_rb, rsz, cudaHostAllocDefault) == cudaSuccess;
        if (ok) {
            // a recorded event for the first wait on each slot
            ok = cudaEventRecord(sl.out_done, p->s_out) == cudaSuccess;
            sl.jobs.reserve(cfg->max_descs);
        }
    }
    if (!ok) {
        release(p);
        return STEGO_E_CUDA;
    }
    *out = p;
    return STEGO_OK;
}

int stego_pipeline_embed(stego_pipeline *p, const stego_host_job *jobs, uint32_t n,
                         stego_result *results, stego_result *readback_results, uint32_t flags)
{
    stego::Trace trace_("stego_pipeline_embed");
    return run(p, jobs, n, results, readback_results, flags, true);
}

int stego_pipeline_extract(stego_pipeline *p, const stego_host_job *jobs, uint32_t n,
                           stego_result *results)
{
    stego::Trace trace_("stego_pipeline_extract");
    return run(p, jobs, n, results, nullptr, 0, false);
}

int stego_pipeline_destroy(stego_pipeline *p)
{
    if (!p)
        return STEGO_OK;
    cudaStreamSynchronize(p->s_in);
    cudaStreamSynchronize(p->s_comp);
    cudaStreamSynchronize(p->s_out);
    release(p);
    return STEGO_OK;
}

} // extern "C"

static_assert(sizeof(stego_host_job) == 80, "stego_host_job layout");
static_assert(sizeof(stego_pipeline_config) == 56, "stego_pipeline_config layout");
