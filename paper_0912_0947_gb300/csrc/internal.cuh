// internal.cuh -- declarations shared by the CUDA translation units of
// libstego.so (not part of the public ABI; see include/stego.h).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "stego.h"

namespace stego {

// A named range on the calling host thread for profilers and tracers that
// attach through NVTX (nothing but a pointer test when none is attached):
// every entry point, batch and pipeline chunk opens one.
struct Trace {
    explicit Trace(const char *name) { nvtxRangePushA(name); }
    ~Trace() { nvtxRangePop(); }
    Trace(const Trace &) = delete;
    Trace &operator=(const Trace &) = delete;
};

// ---------------------------------------------------------------------------
// Launch shapes
// ---------------------------------------------------------------------------

struct Shape {
    int threads;         // threads per CTA
    int vec;             // 16-byte vectors per thread per loop iteration
    int ctas_per_sm;     // 0 = as many as occupancy allows
    uint32_t tile_bytes; // batched: cover bytes per tile; single-cover STREAM1:
                         // 0 = register kernels, else ring bytes per CTA of
                         // the shared-memory staged kernels
};

// The shape installed for `op`, with the fields of `override_` (if non-null
// and non-zero) taking precedence.
Shape shape_for(int op, const stego_tune *override_);

// Field ranges of a caller-supplied launch shape are valid.
bool tune_ok(const stego_tune *t);

// Number of SMs of the current device (cached per device).
int sm_count();

// Identity of the current CUDA context (process-unique, never reused), or 0
// when it cannot be read.  Caches of device addresses (module globals) are
// keyed on it: a device reset gives the device a new context, in which the
// library's module is loaded again.
unsigned long long context_id();

// Persistent grid: min(ceil(units / units_per_cta), SMs * resident CTAs).
// `kernel` is the __global__ function (for the occupancy query).
int persistent_grid(const void *kernel, int threads, size_t smem, int ctas_per_sm,
                    uint64_t units, uint64_t units_per_cta);

// Programmatic dependent launch: the kernel may be launched while the kernel
// before it in the stream is still finishing (its CTAs then wait on the SMs
// instead of behind the launch).  Only for kernels that call
// grid_dependency_wait() before their first global memory access.
cudaError_t launch_dependent(const void *kernel, dim3 grid, dim3 block, void **args,
                             size_t smem, cudaStream_t s);

// Returns once the grid before this one in the stream has completed and its
// memory operations are visible (at once when there is none, or when the
// launch was an ordinary one).
__device__ __forceinline__ void grid_dependency_wait()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Lets the next kernel in the stream that was launched with
// launch_dependent start launching (it still waits for this grid's end in
// its own grid_dependency_wait()).
__device__ __forceinline__ void allow_dependents()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// ---------------------------------------------------------------------------
// Fused statistics without a zeroing copy
// ---------------------------------------------------------------------------

// Accumulator of one launch's changed-byte count and squared error, one per
// stream (a static device array, zero at load).  Every CTA adds its partial
// totals and then takes a ticket; the CTA with the last ticket moves the
// totals into the result and clears the slot for the stream's next launch.
struct StatSlot {
    unsigned long long changed;
    unsigned long long sse;
    unsigned int arrived;
    unsigned int pad;
    unsigned long long pad2;
};

// The slot of stream s on the current device, or nullptr: then the caller
// zeroes res->changed/sse before the launch and the CTAs add into them.
// Slots are keyed by the stream's ID (cudaStreamGetId), which the runtime
// never reuses, so a stream created after another was destroyed never
// shares the old stream's slot (whose last launch may still be running).
// nullptr for streams being captured into a graph (a replay may run beside
// direct calls on the same stream), for the per-thread default stream
// (one handle, several streams) and once every slot is taken (256 streams
// per device; slots are never handed back, the later streams take the
// zeroing path).
StatSlot *stats_slot(cudaStream_t s);

// ---------------------------------------------------------------------------
// Launchers (all stream-ordered, no synchronisation).  They return the CUDA
// error of the launch.  `res` (nullable) receives msg_bytes = res_msg_bytes
// and status STEGO_OK from block 0 of the launch; with `stats`, res->changed
// and res->sse accumulate the changed-byte count and squared error and must
// have been zeroed by the caller.
// ---------------------------------------------------------------------------

// STREAM1 embed.  n_bytes: bytes written (C out of place, T in place).
// t_bytes: carrying bytes T = 8 * slen, slen = stream length in bytes
// (message plus 4 header bytes when `header`).  nbits: the header value.
cudaError_t s1_embed(const uint8_t *cover, uint8_t *stego, uint64_t n_bytes, uint64_t t_bytes,
                     const uint8_t *msg, uint64_t slen, bool header, uint32_t nbits, bool stats,
                     stego_result *res, uint64_t res_msg_bytes, const Shape &sh, cudaStream_t s,
                     StatSlot *slot = nullptr);

// STREAM1 extract.  With `header`, the length comes from the stego and all
// fields of `res` (required) are written by block 0; otherwise raw_len bytes
// are extracted and `res` is optional.
cudaError_t s1_extract(const uint8_t *st, uint64_t C, uint8_t *msg, uint64_t cap,
                       uint64_t raw_len, bool header, stego_result *res, const Shape &sh,
                       cudaStream_t s);

// PAPER2 (Sections VI/VII), N > 0.  The embed writes only the 4N plane bytes
// it carries: out of place the caller has copied the cover into stego first.
cudaError_t p2_embed(const uint8_t *cover, uint8_t *stego, const stego_geom &g,
                     const uint8_t *msg, uint64_t N, bool stats, stego_result *res,
                     const Shape &sh, cudaStream_t s, StatSlot *slot = nullptr);
cudaError_t p2_extract(const uint8_t *st, const stego_geom &g, uint8_t *msg, uint64_t N,
                       stego_result *res, const Shape &sh, cudaStream_t s);

// PAPER2 out of place in one pass (copy and embed fused); usable when
// p2_fused_ok: distinct 16-byte aligned buffers, 1, 3 or 4 channels and
// 16-byte aligned rows.  N may be 0 (a copy).
bool p2_fused_ok(const uint8_t *cover, const uint8_t *stego, const stego_geom &g);
cudaError_t p2_embed_fused(const uint8_t *cover, uint8_t *stego, const stego_geom &g,
                           const uint8_t *msg, uint64_t N, bool stats, stego_result *res,
                           const Shape &sh, cudaStream_t s, StatSlot *slot = nullptr);

// STREAM1 with k = 1..4 bits per carrying byte, over all bytes or one plane
// (k >= 2 or plane_only; k = 1 over all bytes is s1_embed).
cudaError_t sk_embed(const uint8_t *cover, uint8_t *stego, uint64_t C, uint32_t k, bool plane_only,
                     const stego_geom *g, const uint8_t *msg, uint64_t m, bool header,
                     bool stats, stego_result *res, const Shape &sh, cudaStream_t s,
                     StatSlot *slot = nullptr);
cudaError_t sk_extract(const uint8_t *st, uint64_t C, uint32_t k, bool plane_only,
                       const stego_geom *g, uint8_t *msg, uint64_t cap, uint64_t raw_len,
                       bool header, stego_result *res, const Shape &sh, cudaStream_t s);

// STREAM1 extraction with the message packed by warp ballots (one stego
// byte per lane; ballot.cu); same arguments and results as s1_extract.
cudaError_t s1_extract_ballot(const uint8_t *st, uint64_t C, uint8_t *msg, uint64_t cap,
                              uint64_t raw_len, bool header, stego_result *res, const Shape &sh,
                              cudaStream_t s);

// STREAM1 kernels staged through shared memory with bulk asynchronous
// copies (bulk.cu); same arguments and results as s1_embed / s1_extract.
// Usable with 16-byte aligned buffers when bulk_stages(sh) >= 2: a shape
// with tile_bytes = ring bytes per CTA, tiles of threads * 16 * vec bytes.
uint32_t bulk_stages(const Shape &sh);
cudaError_t s1_embed_bulk(const uint8_t *cover, uint8_t *stego, uint64_t n_bytes,
                          uint64_t t_bytes, const uint8_t *msg, uint64_t slen, bool header,
                          uint32_t nbits, bool stats, stego_result *res, uint64_t res_msg_bytes,
                          const Shape &sh, cudaStream_t s, StatSlot *slot = nullptr);
cudaError_t s1_extract_bulk(const uint8_t *st, uint64_t C, uint8_t *msg, uint64_t cap,
                            uint64_t raw_len, bool header, stego_result *res, const Shape &sh,
                            cudaStream_t s);

// Changed-byte count and SSE of two arrays into out2[0..1] (zeroed by the
// caller).
cudaError_t changed_bytes(const uint8_t *a, const uint8_t *b, uint64_t n,
                          unsigned long long *out2, const Shape &sh, cudaStream_t s);

// One thread writes a whole result (calls that launch no other kernel).
cudaError_t write_result(stego_result *res, uint64_t msg_bytes, int status, cudaStream_t s);

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------

// Adds (a, b) of every thread of the block into out[0], out[1] with one pair
// of 64-bit atomics per block.  All threads of the block must call it.
__device__ __forceinline__ void block_add2(unsigned long long a, unsigned long long b,
                                           unsigned long long *out)
{
    __shared__ unsigned long long sa[32], sb[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xFFFFFFFFu, a, o);
        b += __shfl_down_sync(0xFFFFFFFFu, b, o);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        sa[w] = a;
        sb[w] = b;
    }
    __syncthreads();
    if (w == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        a = lane < nw ? sa[lane] : 0ull;
        b = lane < nw ? sb[lane] : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(0xFFFFFFFFu, a, o);
            b += __shfl_down_sync(0xFFFFFFFFu, b, o);
        }
        if (lane == 0) {
            if (a)
                atomicAdd(out, a);
            if (b)
                atomicAdd(out + 1, b);
        }
    }
}

// The statistics of a single-cover launch: the block's totals go into
// res->changed/sse (zeroed by the caller) without a slot, or into the slot,
// whose last arriving CTA writes res->changed/sse.  All threads of every
// CTA of the grid must call it once.
__device__ __forceinline__ void block_stats(unsigned long long a, unsigned long long b,
                                            stego_result *res, StatSlot *slot)
{
    if (!slot) {
        block_add2(a, b, reinterpret_cast<unsigned long long *>(&res->changed));
        return;
    }
    __shared__ unsigned long long sa[32], sb[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xFFFFFFFFu, a, o);
        b += __shfl_down_sync(0xFFFFFFFFu, b, o);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        sa[w] = a;
        sb[w] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        a = 0;
        b = 0;
        for (int i = 0; i < nw; ++i) {
            a += sa[i];
            b += sb[i];
        }
        if (a)
            atomicAdd(&slot->changed, a);
        if (b)
            atomicAdd(&slot->sse, b);
        __threadfence(); // the adds are visible before the ticket
        if (atomicAdd(&slot->arrived, 1u) == gridDim.x - 1) {
            __threadfence();
            res->changed = atomicExch(&slot->changed, 0ull);
            res->sse = atomicExch(&slot->sse, 0ull);
            atomicExch(&slot->arrived, 0u);
        }
    }
}

// Changed-byte count and squared error of one 32-bit word pair (four bytes).
__device__ __forceinline__ void word_stats(uint32_t x, uint32_t y, unsigned long long &changed,
                                           unsigned long long &sse)
{
    uint32_t d = x ^ y;
    d |= d >> 4; // fold each byte's eight bits into its bit 0
    d |= d >> 2;
    d |= d >> 1;
    changed += __popc(d & 0x01010101u);
    const uint32_t a = __vabsdiffu4(x, y);
    sse += __dp4a(a, a, 0u);
}

// Warp staging of pixel units (16 pixels of CH channels = CH 16-byte
// vectors): a warp's 32 consecutive units are loaded and stored in memory
// order and exchanged through shared memory, SV = unit_stage_slots<CH>()
// slots per warp.  Vector v of the warp's units sits in slot
// unit_stage_slot<CH>(v); CH = 4 pads one slot per 8 so that both the
// memory-order (v = 32j + lane) and the unit-order (v = CH*lane + q)
// accesses are free of bank conflicts (CH = 3 needs no padding).
template <int CH>
__host__ __device__ constexpr uint32_t unit_stage_slots()
{
    return 32 * CH + (CH == 4 ? 16 : 0);
}

template <int CH>
__device__ __forceinline__ uint32_t unit_stage_slot(uint32_t v)
{
    return CH == 4 ? v + (v >> 3) : v;
}

} // namespace stego

