/*
 * stego.h -- C ABI of the GB300 LSB substitution steganography library
 * (libstego.so, built for sm_103a).
 *
 * The method (Patel, Pradhan and Ambegaokar, "A Novel Approach for
 * Implementing Steganography with Computing Power Obtained by Combining CUDA
 * and MATLAB"): hide a message in the least significant bits of uint8 cover
 * image or video-frame bytes (Section VI, embedding) and read it back
 * (Section VII, extraction).  Two bit layouts are provided:
 *
 *   STEGO_LAYOUT_STREAM1  one bit per cover byte, over the cover bytes in
 *       memory order (row-major, interleaved channels).  The embedded stream
 *       is S = BE32(8*m) || msg with STEGO_HEADER_BE32 (a 32-bit big-endian
 *       count of message bits, then the message), or S = msg without it.
 *       Cover byte k carries bit k of S, bits taken most significant first
 *       within each stream byte:
 *           stego[k] = (cover[k] & 0xFE) | ((S[k/8] >> (7 - k%8)) & 1),
 *       for k < T = 8*|S|; bytes k >= T are the cover's.  This is the
 *       Section VI substitution rule (clear low bits, OR in message bits)
 *       with one bit per byte and a sequential layout.
 *
 *   STEGO_LAYOUT_PAPER2   Sections VI and VII as printed: one colour plane
 *       (Section VI step 2) of an H x W x channels interleaved image, two
 *       bits per cover byte, the message divided greedily among rows with
 *       L = min(remaining, floor(W/4)) bytes per row (Section VII step 4), and
 *       bit pair i (bits 2i..2i+1) of data byte B[j] written to row position
 *       A[L*i + j] (Section VI step 7):
 *           A[L*i + j] = (A[L*i + j] & 0xFC) | ((B[j] >> 2i) & 3).
 *       The length is passed out of band, as the paper's extract(E, N) call
 *       does (Section VIII).
 *
 * Conventions common to every entry point
 *   - Pointers named d_* are device pointers (CUDA global memory of the
 *     current device).  Pointers to stego_geom / stego_tune are host
 *     pointers, read before the call returns.  The caller owns every buffer;
 *     the library allocates no device memory in any call.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *     asynchronous and stream-ordered; none synchronises the device.
 *   - Kernels are launched as programmatic dependent launches: each waits
 *     for the previous grid in the stream before touching memory, and lets
 *     the next grid start launching early.  A caller's own kernel launched
 *     after a call with the programmatic stream serialization attribute must
 *     therefore wait (cudaGridDependencySynchronize / griddepcontrol.wait)
 *     before reading the call's outputs, as any such launch must; ordinary
 *     launches, copies and events see plain stream order.
 *   - Errors detectable from the arguments (null pointers, sizes, capacity,
 *     geometry, flags, overlapping buffers) are returned synchronously and
 *     nothing is launched or written.  Errors that depend on device data (a
 *     malformed header, a message buffer too small for the header's length)
 *     are written to the stego_result status field on the device; in that
 *     case the message buffer is not written.  STEGO_E_CUDA means a CUDA
 *     launch or memset failed (see cudaGetLastError in the caller's runtime).
 *   - Any byte alignment is accepted.  Cover and stego buffers that start on
 *     16-byte boundaries take the vectorised (128-bit) path.
 *   - In-place embedding (d_stego == d_cover) is allowed and then bytes past
 *     the embedded bits are not written.  Any other overlap between the
 *     buffers of one call is STEGO_E_INVAL.
 */
#ifndef STEGO_H
#define STEGO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ */
/* Status codes                                                        */
/* ------------------------------------------------------------------ */
enum stego_status {
    STEGO_OK = 0,
    STEGO_E_INVAL = -1,         /* bad argument, flag, geometry or overlap    */
    STEGO_E_CAPACITY = -2,      /* message does not fit in the cover          */
    STEGO_E_BAD_HEADER = -3,    /* header absent, not whole bytes, too long   */
    STEGO_E_MSG_TOO_SMALL = -4, /* output message buffer smaller than length  */
    STEGO_E_CUDA = -5,          /* a CUDA runtime call failed                 */
    STEGO_E_NOMEM = -6,         /* caller-supplied workspace too small        */
    STEGO_E_TIMEOUT = -7        /* a bounded device-side wait ran out         */
};

/* ------------------------------------------------------------------ */
/* Flags                                                               */
/* ------------------------------------------------------------------ */
#define STEGO_LAYOUT_STREAM1 0x0u
#define STEGO_LAYOUT_PAPER2 0x1u
#define STEGO_LAYOUT_MASK 0xFu
#define STEGO_HEADER_BE32 0x10u /* STREAM1 only: 32-bit big-endian bit count */
#define STEGO_FUSE_STATS 0x20u  /* embed: count changed bytes and SSE      */
/* STREAM1 variants between one bit per byte and Section VI's two:
 *   STEGO_BITS(k), k = 1..4: k low bits of every carrying byte take the next
 *   k stream bits, the first in the field's highest bit (stream bit b goes to
 *   bit k-1-(b mod k) of carrying byte b/k); when 8|S| is not a multiple of
 *   k the last carrying byte changes only its top (8|S| mod k) field bits.
 *   STEGO_PLANE_ONLY: the carrying bytes are the bytes of channel
 *   geom->plane in pixel order (Section VI step 2), carrying byte x being
 *   cover byte x*channels + plane; geom is then required.
 * Without either flag STREAM1 is one bit over every byte in memory order.
 * The batched and serving calls take the default (one bit, all bytes). */
#define STEGO_PLANE_ONLY 0x40u
#define STEGO_BITS_MASK 0x300u
#define STEGO_BITS(k) ((((uint32_t)(k)) - 1u) << 8)

/* Image geometry for STEGO_LAYOUT_PAPER2: `height` rows of `width` pixels
 * with `channels` interleaved uint8 channels; the message goes into channel
 * `plane` (Section VI step 2).  cover_bytes must equal width*height*channels. */
typedef struct stego_geom {
    uint32_t width;
    uint32_t height;
    uint32_t channels;
    uint32_t plane;
} stego_geom;

/* Per-call result, in device memory (32 bytes, 8-byte aligned).
 *   changed    embed with STEGO_FUSE_STATS: number of bytes whose value
 *              changed; otherwise 0.
 *   sse        embed with STEGO_FUSE_STATS: sum over all cover bytes of
 *              (stego - cover)^2 (exact, integer); MSE = sse / cover_bytes and
 *              PSNR = 10 log10(255^2 / MSE), the Section VIII quality figure.
 *   msg_bytes  embed: message bytes embedded; extract: bytes extracted.
 *   status     STEGO_OK or the device-detected error of the call. */
typedef struct stego_result {
    uint64_t changed;
    uint64_t sse;
    uint64_t msg_bytes;
    int32_t status;
    int32_t reserved;
} stego_result;

/* One cover of a batched call (device memory, 72 bytes, 8-byte aligned).
 *   cover        embed: the cover; extract: the stego image to read.
 *   stego        embed: output image (may equal cover); extract: unused.
 *   msg          embed: message to hide (read); extract: output buffer.
 *   cover_bytes  size of cover (and stego) in bytes.
 *   msg_bytes    embed: message length; extract: capacity of msg.
 *   msg_len      extract without a header (raw STREAM1, PAPER2): bytes to
 *                extract; ignored otherwise.
 *   flags        STEGO_LAYOUT_STREAM1 (one bit per byte, with or without
 *                STEGO_HEADER_BE32) or STEGO_LAYOUT_PAPER2; STEGO_FUSE_STATS
 *                is taken from the batched call instead.  The k-bit and
 *                one-plane stream options (STEGO_BITS(k), k > 1, and
 *                STEGO_PLANE_ONLY) are single-cover only: such a
 *                descriptor gets STEGO_E_INVAL in its result.
 *   geom         PAPER2 geometry. */
typedef struct stego_desc {
    const uint8_t *cover;
    uint8_t *stego;
    uint8_t *msg;
    uint64_t cover_bytes;
    uint64_t msg_bytes;
    uint64_t msg_len;
    uint32_t flags;
    uint32_t reserved;
    stego_geom geom;
} stego_desc;

/* Launch shape.  Zero fields take the library's current choice for the
 * operation (installed by stego_set_tune, initially built-in defaults).
 *   threads         threads per CTA (multiple of 32, 64..512)
 *   vec_per_thread  16-byte vectors each thread keeps in flight per loop
 *                   iteration (1, 2, 4 or 8)
 *   ctas_per_sm     resident CTAs per SM of the persistent grid
 *   tile_bytes      a multiple of 4096.  Batched calls: cover bytes per work
 *                   tile (at least 4096).  Single-cover one-bit STREAM1
 *                   embed and extract on 16-byte aligned buffers: 0 selects
 *                   the register-streaming kernels; otherwise the kernels
 *                   staged through shared memory by bulk asynchronous
 *                   copies, with a ring of tile_bytes bytes per CTA cut into
 *                   stages of threads * 16 * vec_per_thread bytes (2 to 8
 *                   stages, at most 192 KiB; a ring smaller than two stages
 *                   selects the register kernels).  For STEGO_OP_EMBED and
 *                   STEGO_OP_EXTRACT, stego_set_tune installs tile_bytes as
 *                   given, 0 included. */
typedef struct stego_tune {
    uint32_t threads;
    uint32_t vec_per_thread;
    uint32_t ctas_per_sm;
    uint32_t tile_bytes;
} stego_tune;

enum stego_op {
    STEGO_OP_EMBED = 0,
    STEGO_OP_EXTRACT = 1,
    STEGO_OP_CHANGED = 2,
    STEGO_OP_EMBED_BATCHED = 3,
    STEGO_OP_EXTRACT_BATCHED = 4,
    STEGO_OP_COUNT = 5
};

/* Library version (major*10000 + minor*100 + patch). */
int stego_version(void);

/* Human-readable name of a status code (static storage). */
const char *stego_strerror(int status);

/* Largest message (bytes) that fits a cover of `cover_bytes`:
 *   STREAM1 with header: floor(k*Cc/8) - 4 (at least 0, at most 2^29 - 1;
 *                        Cc = carrying bytes: cover_bytes, or width*height
 *                        with STEGO_PLANE_ONLY; a cover whose k*Cc is under
 *                        32 bits cannot hold the header, so even an empty
 *                        message is STEGO_E_CAPACITY there);
 *   STREAM1 raw:        floor(k*Cc/8);
 *   PAPER2:             floor(W/4) * H   (Section VI step 5: 4*|B| <= |A|).
 * geom is required for PAPER2 and STEGO_PLANE_ONLY and ignored otherwise.
 * Writes *out_msg_bytes.
 * Returns STEGO_OK or STEGO_E_INVAL. */
int stego_capacity(uint64_t cover_bytes, const stego_geom *geom, uint32_t flags,
                   uint64_t *out_msg_bytes);

/* Embed (Section VI).  Writes cover_bytes bytes of d_stego (out of place) or,
 * in place, the T = 8*|S| carrying bytes (STREAM1) / the 4*msg_bytes plane
 * bytes (PAPER2; with 1, 3 or 4 channels, rows of whole 16-byte vectors and
 * a 16-byte aligned buffer whole 16-pixel groups are rewritten, the bytes
 * outside the plane's carrying bytes with their own values: those groups
 * holding carrying pixels, in a batched call every group of the carrying
 * rows).  Bytes that do not carry the message keep their values.
 *   d_cover, d_stego  cover and output image, cover_bytes each.
 *   d_msg, msg_bytes  message (may be NULL when msg_bytes == 0).
 *   geom              PAPER2 geometry (host pointer) or NULL for STREAM1.
 *   flags             layout | STEGO_HEADER_BE32 (STREAM1) | STEGO_FUSE_STATS.
 *   d_result          optional; required with STEGO_FUSE_STATS.  Filled with
 *                     changed/sse (if fused), msg_bytes and status STEGO_OK.
 * Synchronous errors: STEGO_E_INVAL, STEGO_E_CAPACITY (message too long for
 * the cover; nothing written), STEGO_E_CUDA. */
int stego_embed(const uint8_t *d_cover, uint8_t *d_stego, uint64_t cover_bytes,
                const uint8_t *d_msg, uint64_t msg_bytes, const stego_geom *geom,
                uint32_t flags, stego_result *d_result, void *stream);

/* Extract (Section VII).
 *   d_stego, cover_bytes  the stego image.
 *   d_msg, msg_cap        output buffer and its capacity in bytes.
 *   msg_len               bytes to extract without a header (raw STREAM1 and
 *                         PAPER2, the paper's out-of-band N); ignored with
 *                         STEGO_HEADER_BE32.
 *   d_result              required with STEGO_HEADER_BE32 (the length and
 *                         status come from the device); optional otherwise.
 * With the header, the 32-bit count is read from the LSBs of bytes 0..31 and
 * is rejected on the device (status STEGO_E_BAD_HEADER) when the stego is
 * shorter than 32 bytes, the count is not a multiple of 8 or 32 + count
 * exceeds cover_bytes; STEGO_E_MSG_TOO_SMALL when count/8 > msg_cap.  On any
 * device-side error d_msg is not written and msg_bytes is 0.
 * Without the header the bounds are checked on the host: STEGO_E_CAPACITY
 * when msg_len exceeds stego_capacity, STEGO_E_MSG_TOO_SMALL when
 * msg_len > msg_cap. */
int stego_extract(const uint8_t *d_stego, uint64_t cover_bytes, uint8_t *d_msg,
                  uint64_t msg_cap, uint64_t msg_len, const stego_geom *geom,
                  uint32_t flags, stego_result *d_result, void *stream);

/* stego_extract for the one-bit stream layout (STEGO_LAYOUT_STREAM1, one bit
 * per byte, all bytes; other flags give STEGO_E_INVAL) computed by a kernel
 * that packs the message with warp ballots: lane l of a warp loads stego
 * byte 32w + l and one ballot of the 32 LSBs is message word w.  Same
 * arguments, results and errors as stego_extract; the paper has no
 * counterpart.  It exists to compare the ballot gather with stego_extract's
 * kernel (16 stego bytes per lane from one 128-bit load, one multiply per
 * four bytes), which is about 4x faster on a 201 MB stego. */
int stego_extract_ballot(const uint8_t *d_stego, uint64_t cover_bytes, uint8_t *d_msg,
                         uint64_t msg_cap, uint64_t msg_len, const stego_geom *geom,
                         uint32_t flags, stego_result *d_result, void *stream);

/* Changed-byte count and squared error of two equal-length byte arrays
 * (Section VIII reports PSNR of stego against cover).
 *   d_out2[0] = #{k : a[k] != b[k]},  d_out2[1] = sum (a[k] - b[k])^2.
 * d_out2 is device memory, two uint64 (8-byte aligned). */
int stego_changed_bytes(const uint8_t *d_a, const uint8_t *d_b, uint64_t n,
                        uint64_t *d_out2, void *stream);

/* Device workspace (bytes) a batched call over n descriptors needs. */
uint64_t stego_batched_workspace_bytes(uint32_t n);

/* Batched embed: every descriptor of d_descs[0..n) (device memory) in one
 * persistent launch that claims fixed-size tiles of the covers from a work
 * counter.  The paper repeats the per-row routine over rows and video frames
 * (Section VI, last paragraph; "image/video frames", Section III); here all
 * covers and frames of a batch are one launch.
 *   d_results  n results (device), one per descriptor: status, msg_bytes and,
 *              with STEGO_FUSE_STATS in `flags`, changed and sse.
 *   flags      STEGO_FUSE_STATS or 0 (per-cover layout flags are in the
 *              descriptors).
 *   tune       optional launch shape (host pointer); NULL = current choice.
 *   d_ws       caller-owned device workspace of ws_bytes >=
 *              stego_batched_workspace_bytes(n), 16-byte aligned.  It is
 *              scratch: its contents on entry do not matter and on return
 *              are unspecified.
 * Both layouts may be mixed in one batch.  One-bit stream covers are cut
 * into tiles of cover bytes; paper-layout covers into tiles of whole rows
 * (out of place: rows are copied, then their plane bytes rewritten).
 * Descriptor errors (capacity, geometry, overlap) are per cover: that
 * cover's status is set and its output is not written; other covers
 * proceed.  Returns STEGO_E_NOMEM when ws_bytes is too small. */
int stego_embed_batched(const stego_desc *d_descs, uint32_t n, stego_result *d_results,
                        uint32_t flags, const stego_tune *tune, void *d_ws,
                        uint64_t ws_bytes, void *stream);

/* Batched extract (Section VII); same arguments.  Each descriptor's cover is
 * the stego image and msg its output buffer of msg_bytes capacity. */
int stego_extract_batched(const stego_desc *d_descs, uint32_t n, stego_result *d_results,
                          uint32_t flags, const stego_tune *tune, void *d_ws,
                          uint64_t ws_bytes, void *stream);

/* Batched embed that allocates nothing, for callers that cannot call
 * cudaMalloc (a host program with no device allocator of its own, or one that
 * may not add cudaMalloc's implicit device synchronisation to a per-request
 * path).  The paper has no counterpart; it is stego_embed_batched with the
 * workspace taken from a scratch array inside the library instead of d_ws.
 *   n  at most STEGO_NOALLOC_MAX_DESCS; larger batches return
 *      STEGO_E_NOMEM and nothing is launched.  Bad flags or a bad tune are
 *      reported first (STEGO_E_INVAL), as stego_embed_batched does.
 * Other arguments, results and per-cover errors as for stego_embed_batched.
 * The scratch array (about 640 KiB) is one per GPU, held by every GPU that
 * loads the library until the process exits.  The first call on a device
 * sets up that device (it looks up the array's device address with
 * cudaGetSymbolAddress); make that first call before any stream capture.
 * After a cudaDeviceReset the next call sets the device up again (the
 * address is kept per device together with the identity of the context it
 * belongs to).
 * Every call on a device shares the one array: calls whose work overlaps on
 * the GPU (different streams, or different host threads) race and must be
 * serialised by the caller, e.g. by issuing them on one stream.  Each call
 * rewrites all the scratch it uses, so no clearing is needed between calls. */
#define STEGO_NOALLOC_MAX_DESCS 8192u
int stego_embed_batched_noalloc(const stego_desc *d_descs, uint32_t n, stego_result *d_results,
                                uint32_t flags, const stego_tune *tune, void *stream);

/* CUDA graph of one batched call.  The descriptors, results and workspace
 * are captured by address: fill the same device arrays with new descriptors
 * (same n) and replay, which re-runs the three launches of the call without
 * host-side launch overhead.  The graph object (and its instantiation) is
 * the only thing these functions create; stego_graph_destroy releases it.
 *   op  STEGO_OP_EMBED_BATCHED or STEGO_OP_EXTRACT_BATCHED.
 * Capture uses a private stream in thread-local capture mode, so it does not
 * disturb work the caller has in flight. */
typedef struct stego_graph stego_graph;
int stego_graph_capture_batched(int op, const stego_desc *d_descs, uint32_t n,
                                stego_result *d_results, uint32_t flags, const stego_tune *tune,
                                void *d_ws, uint64_t ws_bytes, stego_graph **out);
int stego_graph_launch(stego_graph *g, void *stream);
int stego_graph_destroy(stego_graph *g);

/* ------------------------------------------------------------------ */
/* Serving: continuous batching of embed / extract requests            */
/* ------------------------------------------------------------------ */
/* A server owns one dispatcher thread and `slots` CUDA streams.  Requests
 * of mixed sizes are queued by stego_server_submit (any thread).  Whenever a
 * slot is free the dispatcher admits queued requests in arrival order while
 * the sum of their working-set bytes (embed: 2*cover_bytes + msg_bytes;
 * extract: cover_bytes + msg_bytes) stays within budget_bytes, up to
 * max_batch requests, and launches them as one stego_embed_batched plus one
 * stego_extract_batched on that slot's stream; the batch's stream-layout
 * requests with STEGO_BITS(k), k > 1, or STEGO_PLANE_ONLY (which the
 * batched kernels do not take) follow as stego_embed / stego_extract calls
 * on the same stream, a request they refuse completing with that status.
 * Requests arriving while
 * batches run are admitted into the next free slot as soon as budget frees
 * up, so batches overlap on the device.  A request whose own bytes exceed
 * the budget completes at once with STEGO_E_NOMEM; an unknown op with
 * STEGO_E_INVAL.  This is the paper's per-row / per-frame call repeated
 * (Section VI, last paragraph) turned into a request stream.
 * Buffers named in requests are caller-owned, device-accessible, and must
 * stay valid until the request's completion has been returned. */
typedef struct stego_server stego_server;

typedef struct stego_server_config {
    uint32_t slots;        /* batches in flight at once (1..16)             */
    uint32_t max_batch;    /* requests per batch (1..8192)                  */
    uint64_t budget_bytes; /* in-flight working-set budget, bytes           */
    stego_tune tune_embed; /* launch shapes of the batched calls (zeros =   */
    stego_tune tune_extract; /*  the installed choice)                      */
} stego_server_config;     /* 48 bytes */

typedef struct stego_request {
    uint32_t op;           /* STEGO_OP_EMBED or STEGO_OP_EXTRACT            */
    uint32_t flags;        /* STEGO_LAYOUT_STREAM1 [| STEGO_HEADER_BE32]    */
                           /* [| STEGO_BITS(k)] [| STEGO_PLANE_ONLY, with   */
                           /* geom] or STEGO_LAYOUT_PAPER2 (with geom);     */
                           /* k > 1 and one-plane requests run as single-   */
                           /* cover calls inside their batch                */
    const uint8_t *cover;  /* embed: cover; extract: stego image            */
    uint8_t *stego;        /* embed: output image                           */
    uint8_t *msg;          /* embed: message (read); extract: output buffer */
    uint64_t cover_bytes;
    uint64_t msg_bytes;    /* embed: length; extract: capacity of msg       */
    uint64_t msg_len;      /* extract without a header: bytes to extract    */
    uint64_t tag;          /* returned in the completion                    */
    stego_geom geom;       /* PAPER2 / STEGO_PLANE_ONLY geometry            */
} stego_request;           /* 80 bytes */

typedef struct stego_completion {
    uint64_t tag;
    uint64_t changed;      /* embed: changed bytes (stats always fused)     */
    uint64_t sse;          /* embed: squared error                          */
    uint64_t msg_bytes;    /* embedded / extracted message bytes            */
    int32_t status;        /* STEGO_OK or the request's error               */
    int32_t batch_size;    /* requests in the batch that carried it         */
    double t_submit;       /* server clock, seconds: queued (open loop: the */
    double t_dispatch;     /*   scheduled arrival), launched, and seen done */
    double t_done;
} stego_completion;        /* 64 bytes */

/* Device arena (bytes) a server with this configuration needs: per slot its
 * descriptors, results and batched workspaces.  0 for an invalid config. */
uint64_t stego_server_arena_bytes(const stego_server_config *cfg);

/* Creates a server on the current device.  d_arena: caller-owned device
 * memory of arena_bytes >= stego_server_arena_bytes(cfg), 256-byte aligned,
 * used until stego_server_destroy.  The server allocates no device memory;
 * it allocates its pinned host staging (descriptors and results) here. */
int stego_server_create(const stego_server_config *cfg, void *d_arena, uint64_t arena_bytes,
                        stego_server **out);

/* Queues n requests (copied); thread-safe. */
int stego_server_submit(stego_server *s, const stego_request *reqs, uint32_t n);

/* Moves up to max finished completions into out; *n_out = how many. */
int stego_server_poll(stego_server *s, stego_completion *out, uint32_t max, uint32_t *n_out);

/* Waits until every submitted request has completed (their completions stay
 * queued for stego_server_poll); STEGO_E_TIMEOUT after timeout_s seconds. */
int stego_server_drain(stego_server *s, double timeout_s);

/* Open-loop load: the calling thread submits reqs[i] at arrival_s[i]
 * seconds after the call starts (server clock), then waits for all of them
 * (at most timeout_s) and writes completion i to out[i] (tags are set to i;
 * latency counts from the scheduled arrival).  The server must be idle. */
int stego_server_run_open_loop(stego_server *s, const stego_request *reqs,
                               const double *arrival_s, uint32_t n, stego_completion *out,
                               double timeout_s);

/* Seconds since the server was created; batches launched, requests
 * outstanding and the largest in-flight working set admitted so far (any
 * out pointer may be NULL). */
double stego_server_clock(stego_server *s);
int stego_server_stats(stego_server *s, uint64_t *batches, uint64_t *outstanding,
                       uint64_t *peak_in_flight_bytes);

/* Finishes queued and in-flight work, stops the dispatcher, frees the
 * server (not the arena). */
int stego_server_destroy(stego_server *s);

/* ------------------------------------------------------------------ */
/* Host-resident covers: overlapped copy-in, kernels and copy-out       */
/* ------------------------------------------------------------------ */
/* The paper's gateway (Section V) copies the image into device memory,
 * runs the kernel and copies the result back.  A pipeline does that for a
 * batch of covers that live in host memory: it cuts the batch into chunks
 * that fit one device staging slot and runs chunk k on slot k mod `slots`
 * as three stages on three streams of its own (host -> slot copies; one
 * batched embed in place on the slot, plus one batched extract of the new
 * stegos for jobs that ask for a read-back, or one batched extract; slot ->
 * host copies), so that with two or more slots the copies of neighbouring
 * chunks in both directions overlap the kernels.  Jobs that reuse nothing
 * on the device can instead be zero copy (see STEGO_PIPE_AUTO).  Every
 * calculation runs in the batched kernels on the device; the host only
 * plans the chunks and issues copies.
 *
 * Host buffers should be pinned (cudaHostAlloc / cudaHostRegister) for the
 * copies to overlap.  An extraction's message is written by the kernel
 * straight into the job's host buffer, which must therefore be memory the
 * device may dereference (pinned and mapped, the usual case with unified
 * addressing, or any host memory on devices with pageable memory access);
 * otherwise that job gets STEGO_E_INVAL. */
typedef struct stego_pipeline stego_pipeline;

/* Transport of a pipeline's jobs (stego_pipeline_config.mode).
 *   STEGO_PIPE_AUTO    jobs that reuse data on the device (an embed whose
 *                      stego is read back) are staged through the slots;
 *                      every other job is zero copy: the batched kernels
 *                      read and write its host buffers over the CPU-GPU
 *                      link (an extraction then reads only the stego's
 *                      carrying bytes).  Zero copy needs buffers the device
 *                      may dereference; a job whose buffers are not is
 *                      staged.
 *   STEGO_PIPE_STAGED  every job is staged: covers and messages copied in,
 *                      stegos copied back, by the copy engines (extracted
 *                      messages are still written by the kernel). */
#define STEGO_PIPE_AUTO 0u
#define STEGO_PIPE_STAGED 1u

typedef struct stego_pipeline_config {
    uint32_t slots;        /* device staging slots (1..8); 2 or 3 overlap   */
    uint32_t max_descs;    /* covers per chunk (1..8192)                    */
    uint64_t slot_bytes;   /* data bytes per slot (>= 4096) for the staged  */
                           /* covers, messages and read-backs of a chunk    */
    uint32_t mode;         /* STEGO_PIPE_AUTO or STEGO_PIPE_STAGED          */
    uint32_t reserved;     /* 0                                             */
    stego_tune tune_embed; /* launch shapes of the batched calls (zeros =   */
    stego_tune tune_extract; /*  the installed choice)                      */
} stego_pipeline_config;   /* 56 bytes */

/* One host-resident job (host memory, 80 bytes).
 *   cover        embed: the cover; extract: the stego image.
 *   stego        embed: output image; may equal cover (then only the bytes
 *                that can carry the message are copied in and back: the
 *                first 8*|S| bytes of the stream layout, the carrying rows
 *                of the paper layout).
 *   msg          embed: the message (read); extract: output buffer.
 *   readback     embed, optional (NULL = none): receives msg_bytes bytes, the
 *                extraction of the new stego, made on the device before it
 *                is copied back (a sender's check that the stego decodes).
 *   cover_bytes, msg_bytes, msg_len, flags, geom  as in stego_desc. */
typedef struct stego_host_job {
    const uint8_t *cover;
    uint8_t *stego;
    uint8_t *msg;
    uint8_t *readback;
    uint64_t cover_bytes;
    uint64_t msg_bytes;
    uint64_t msg_len;
    uint32_t flags;
    uint32_t reserved;
    stego_geom geom;
} stego_host_job;

/* Device arena (bytes) a pipeline with this configuration needs: per slot
 * its descriptors, results, batched workspace and data area.  0 for an
 * invalid configuration. */
uint64_t stego_pipeline_arena_bytes(const stego_pipeline_config *cfg);

/* Creates a pipeline on the current device.  d_arena: caller-owned device
 * memory of arena_bytes >= stego_pipeline_arena_bytes(cfg), 256-byte
 * aligned, used until stego_pipeline_destroy.  The pipeline allocates no
 * device memory; it creates three streams and allocates pinned host staging
 * for descriptors and results here.  One call at a time per pipeline. */
int stego_pipeline_create(const stego_pipeline_config *cfg, void *d_arena, uint64_t arena_bytes,
                          stego_pipeline **out);

/* Embeds jobs[0..n) (host array) and returns when every output is in host
 * memory.  results (host, n): per job, as stego_embed_batched's results.
 * readback_results (host, n, optional): per job the read-back extraction's
 * result (zeros for jobs without a read-back); on a read-back error the
 * readback buffer's contents are unspecified.  flags: STEGO_FUSE_STATS or 0.
 * Per-job argument errors (those of stego_embed_batched, plus
 * STEGO_E_NOMEM for a job that does not fit one slot: it needs cover_bytes
 * + msg_bytes + 1280 bytes, plus msg_bytes rounded up to 256 with a
 * read-back; an extraction needs cover_bytes + 768) are that job's status;
 * its stego is not written and the other jobs proceed.  Returns STEGO_OK,
 * STEGO_E_INVAL or STEGO_E_CUDA (then outputs and results are
 * unspecified). */
int stego_pipeline_embed(stego_pipeline *p, const stego_host_job *jobs, uint32_t n,
                         stego_result *results, stego_result *readback_results, uint32_t flags);

/* Extracts jobs[0..n) (host array; cover = the stego image, msg = output of
 * msg_bytes capacity) and returns when every message is in host memory;
 * results as stego_extract_batched's (STEGO_E_NOMEM for a job that does not
 * fit one slot).  Device-detected errors (header) leave that job's message
 * buffer unwritten. */
int stego_pipeline_extract(stego_pipeline *p, const stego_host_job *jobs, uint32_t n,
                           stego_result *results);

/* Waits for the pipeline's streams, destroys them and frees its host
 * staging (not the arena). */
int stego_pipeline_destroy(stego_pipeline *p);

/* ------------------------------------------------------------------ */
/* Several GPUs: splitting a batch by byte volume                       */
/* ------------------------------------------------------------------ */
/* Covers are independent (the paper repeats its routine per row and per
 * frame, Section VI, last paragraph), so a batch shards across `world` GPUs
 * with no exchange step: each GPU runs the batched calls on its own covers
 * and only the per-cover results are gathered.  This call assigns covers
 * to GPUs by byte volume: covers in decreasing size (ties by index), each
 * to the GPU with the fewest bytes so far (ties to the lowest rank), so
 * every GPU ends within one cover's bytes of every other.  Host only: no
 * CUDA call, no device memory.
 *   bytes       host array of n cover sizes (the work of each cover).
 *   rank_of     host array of n: the GPU (0..world-1) of each cover.
 *   rank_bytes  optional host array of world: bytes assigned to each GPU.
 * Returns STEGO_OK, or STEGO_E_INVAL for world == 0, world > 65536 or a
 * null array with n > 0. */
int stego_partition(const uint64_t *bytes, uint32_t n, uint32_t world, uint32_t *rank_of,
                    uint64_t *rank_bytes);

/* Where a buffer lives, as the CUDA runtime of the current device reports
 * it, and whether this library's kernels may read and write it directly.
 *   *kind: STEGO_MEM_PAGEABLE (ordinary host memory), STEGO_MEM_PINNED
 *          (page-locked host memory), STEGO_MEM_DEVICE, STEGO_MEM_MANAGED.
 *   *device_accessible: 1 when a kernel may dereference p itself: device
 *          and managed memory, pinned host memory mapped at the same address
 *          (the usual case with unified addressing; the kernel then reads
 *          and writes host memory over the CPU-GPU link), and pageable host
 *          memory only when the device reports pageable-memory access.
 * Every entry point accepts device-accessible pointers of any kind; this
 * call lets a caller check a host buffer before passing it.
 * Returns STEGO_OK or STEGO_E_CUDA. */
#define STEGO_MEM_PAGEABLE 0
#define STEGO_MEM_PINNED 1
#define STEGO_MEM_DEVICE 2
#define STEGO_MEM_MANAGED 3
int stego_pointer_kind(const void *p, int *kind, int *device_accessible);

/* Test hook for the bounded device-side waits (failure detection).  The
 * paper has no counterpart.  The shared-memory staged kernels (selected by
 * a nonzero tile_bytes for STEGO_OP_EMBED / STEGO_OP_EXTRACT) wait on
 * mbarriers for their bulk copies; every wait is bounded, and a CTA whose
 * wait runs out waits for its copies still in flight, writes
 * STEGO_E_TIMEOUT into the call's stego_result status and returns, leaving
 * the context usable.  This call sets, for launches made after it in this
 * process:
 *   limit_ns          the bound of the pipeline's waits (0 = the default,
 *                     one second; the wait for copies in flight after a
 *                     timeout always keeps the default);
 *   withhold_arrival  1: each stage's barrier expects one arrival more than
 *                     the pipeline gives, so every CTA's first wait runs out
 *                     after limit_ns (a flag that nothing sets); the CTA
 *                     gives the missing arrival while draining, so its copies
 *                     are still waited for.  No output byte is then written
 *                     (the message buffer of an extract, the stego of an
 *                     embed).  0: normal operation.
 * On STEGO_E_TIMEOUT the outputs are otherwise unspecified (CTAs whose waits
 * completed may have written their parts).  Returns STEGO_OK, or
 * STEGO_E_INVAL for withhold_arrival > 1. */
int stego_test_bounded_wait(uint64_t limit_ns, uint32_t withhold_arrival);

/* Install / read the launch shape used by an operation (enum stego_op) on
 * every device.  Zero fields of `t` keep their built-in defaults.
 * Returns STEGO_E_INVAL for an unknown op or an out-of-range field. */
int stego_set_tune(int op, const stego_tune *t);
int stego_get_tune(int op, stego_tune *out);

#ifdef __cplusplus
}
#endif

#endif /* STEGO_H */
