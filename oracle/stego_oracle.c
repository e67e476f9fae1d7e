/*
 * stego_oracle.c -- CPU oracle for LSB substitution steganography.
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only tests/, the smoke check in
 * __graft_entry__.py and the CPU-baseline leg of bench.py may load this file's
 * library.  It shares no code, header, table or helper with the CUDA path
 * (paper_0912_0947_gb300/csrc); the two are compared on the same seeded inputs.
 *
 * Plain, slow, single-threaded C.  Every loop walks bytes or bits in the order
 * the method states, with no blocking, fusion or reordering, so that a reader
 * can check it against the paper by eye.
 *
 * Two layouts are implemented:
 *
 *  - "stream1": 1-bit LSB substitution over the cover's bytes in memory order
 *    (row-major interleaved channels).  The embedded bit stream is
 *    S = BE32(8*m) || msg (or S = msg without the header); bits are taken
 *    most-significant first within each stream byte, and cover byte k carries
 *    stream bit k.  This is the Section VI substitution (clear the low bits of
 *    a cover byte, OR in message bits) with one bit per byte and the message
 *    laid out sequentially; the length travels in a 32-bit big-endian bit-count
 *    header.
 *
 *  - "streamk": the same stream with k = 1..4 bits per carrying byte, the
 *    carrying bytes being every byte or, as in Section VI step 2, one colour
 *    plane in pixel order (k = 1 over all bytes is "stream1").
 *
 *  - "paper2": the literal algorithm of Section VI (embedding) and Section VII
 *    (extraction): one colour plane, two bits per cover byte, the message
 *    divided greedily among image rows with floor(W/4) bytes per row, and the
 *    i-th bit pair of data byte B[j] written to row position A[L*i + j].
 *
 * Status codes (same numeric values as the library's public status enum; an
 * interface that both sides must agree on, written independently here):
 *    0 ok, -1 invalid argument, -2 capacity exceeded, -3 bad header,
 *   -4 message buffer too small.
 *
 * Parity pins: every function here is pinned by the tests in
 * tests/test_oracle_pins.py (hand-worked examples, exhaustive single-byte
 * tables, brute force on tiny covers, invariants, the Section VIII session
 * shape and the Section VIII PSNR gap).  The absolute PSNR values printed in
 * Section VIII need the paper's cover image, which is not available, so those
 * two numbers are parity unpinned; the gap between them is pinned.
 */
#include <stdint.h>
#include <string.h>

#define OR_OK 0
#define OR_E_INVAL (-1)
#define OR_E_CAPACITY (-2)
#define OR_E_BAD_HEADER (-3)
#define OR_E_MSG_TOO_SMALL (-4)

/* Largest message (bytes) whose bit count fits the 32-bit header. */
#define OR_MAX_HEADER_MSG 0x1FFFFFFFull

/* ------------------------------------------------------------------------ */
/* stream1                                                                   */
/* ------------------------------------------------------------------------ */

/* Byte q of the embedded stream S.  With the header, S starts with the four
 * bytes of the 32-bit bit count 8*m, most significant byte first, and the
 * message follows.  Without the header, S is the message itself. */
static uint8_t stream_byte(const uint8_t *msg, uint64_t m, int header, uint64_t q)
{
    if (!header)
        return msg[q];
    if (q < 4) {
        uint32_t nbits = (uint32_t)(8u * m);
        return (uint8_t)(nbits >> (8u * (3u - (uint32_t)q)));
    }
    return msg[q - 4];
}

/* Embed (Section VI substitution, one bit per cover byte).
 * out may equal cover (in place).  Returns a status; on error nothing is
 * written. */
int oracle_stream1_embed(const uint8_t *cover, uint8_t *out, uint64_t C,
                         const uint8_t *msg, uint64_t m, int header)
{
    uint64_t slen, k;
    if (C > 0 && (cover == 0 || out == 0))
        return OR_E_INVAL;
    if (m > 0 && msg == 0)
        return OR_E_INVAL;
    if (header && m > OR_MAX_HEADER_MSG)
        return OR_E_CAPACITY;
    slen = m + (header ? 4u : 0u);
    /* the stream needs 8*slen cover bytes, one per bit */
    if (slen > C / 8u)
        return OR_E_CAPACITY;

    if (out != cover)
        memcpy(out, cover, (size_t)C);

    for (k = 0; k < 8u * slen; ++k) {
        uint8_t s = stream_byte(msg, m, header, k / 8u);
        uint8_t bit = (uint8_t)((s >> (7u - (uint32_t)(k % 8u))) & 1u);
        out[k] = (uint8_t)((cover[k] & 0xFEu) | bit);
    }
    return OR_OK;
}

/* Extract (Section VII, one bit per cover byte).
 * With the header: read the 32-bit bit count from the LSBs of cover bytes
 * 0..31 (most significant first) and validate it.  Without the header the
 * message length raw_len (bytes) is given by the caller, as the paper passes
 * N to its extraction routine.  On success *out_len is the message length and
 * msg[0..len) is written; on error msg is untouched. */
int oracle_stream1_extract(const uint8_t *st, uint64_t C, uint8_t *msg,
                           uint64_t cap, int header, uint64_t raw_len,
                           uint64_t *out_len)
{
    uint64_t base, len, s;
    int b;
    if (out_len)
        *out_len = 0;
    if (C > 0 && st == 0)
        return OR_E_INVAL;
    if (header) {
        uint64_t nbits = 0, k;
        if (C < 32u)
            return OR_E_BAD_HEADER;
        for (k = 0; k < 32u; ++k)
            nbits |= (uint64_t)(st[k] & 1u) << (31u - (uint32_t)k);
        if (nbits % 8u != 0u)
            return OR_E_BAD_HEADER;
        if (32u + nbits > C)
            return OR_E_BAD_HEADER;
        len = nbits / 8u;
        if (len > cap)
            return OR_E_MSG_TOO_SMALL;
        base = 32u;
    } else {
        len = raw_len;
        if (len > C / 8u)
            return OR_E_CAPACITY;
        if (len > cap)
            return OR_E_MSG_TOO_SMALL;
        base = 0u;
    }
    if (len > 0 && msg == 0)
        return OR_E_INVAL;
    for (s = 0; s < len; ++s) {
        uint8_t v = 0;
        for (b = 0; b < 8; ++b)
            v = (uint8_t)(v | ((st[base + 8u * s + (uint64_t)b] & 1u) << (7 - b)));
        msg[s] = v;
    }
    if (out_len)
        *out_len = len;
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* streamk: k bits per carrying byte, all bytes or one plane                 */
/* ------------------------------------------------------------------------ */

/* The variant space between the one-bit stream and Section VI's two bits per
 * byte (step 7c-f masks k = 2 low bits): k = 1..4 low bits of each carrying
 * byte receive the next k stream bits, the first of them in the field's
 * highest bit.  Stream bit b goes to bit (k - 1 - b mod k) of carrying byte
 * b / k; when 8|S| is not a multiple of k, the last carrying byte changes
 * only its top (8|S| mod k) field bits.  Carrying bytes are every cover byte
 * in memory order (plane_only = 0) or, as in Section VI step 2, only the
 * bytes of one colour plane in pixel order: carrying byte x is cover byte
 * x*channels + plane. */

static uint64_t carrying_index(uint64_t x, int plane_only, uint32_t Cch, uint32_t plane)
{
    return plane_only ? x * Cch + plane : x;
}

static int streamk_args_ok(uint64_t C, uint32_t k, int plane_only, uint32_t W, uint32_t H,
                           uint32_t Cch, uint32_t plane)
{
    if (k < 1 || k > 4)
        return 0;
    if (plane_only && (Cch == 0 || plane >= Cch || (uint64_t)W * H * Cch != C))
        return 0;
    return 1;
}

/* Carrying bytes of the cover. */
static uint64_t carrying_bytes(uint64_t C, int plane_only, uint32_t W, uint32_t H)
{
    return plane_only ? (uint64_t)W * H : C;
}

int oracle_streamk_embed(const uint8_t *cover, uint8_t *out, uint64_t C, uint32_t k,
                         int plane_only, uint32_t W, uint32_t H, uint32_t Cch,
                         uint32_t plane, const uint8_t *msg, uint64_t m, int header)
{
    uint64_t slen, nbits_stream, b;
    if (!streamk_args_ok(C, k, plane_only, W, H, Cch, plane))
        return OR_E_INVAL;
    if (C > 0 && (cover == 0 || out == 0))
        return OR_E_INVAL;
    if (m > 0 && msg == 0)
        return OR_E_INVAL;
    if (header && m > OR_MAX_HEADER_MSG)
        return OR_E_CAPACITY;
    slen = m + (header ? 4u : 0u);
    nbits_stream = 8u * slen;
    /* the stream needs ceil(8|S| / k) carrying bytes */
    if ((nbits_stream + k - 1) / k > carrying_bytes(C, plane_only, W, H))
        return OR_E_CAPACITY;

    if (out != cover)
        memcpy(out, cover, (size_t)C);

    for (b = 0; b < nbits_stream; ++b) {
        uint8_t s = stream_byte(msg, m, header, b / 8u);
        uint8_t bit = (uint8_t)((s >> (7u - (uint32_t)(b % 8u))) & 1u);
        uint64_t x = carrying_index(b / k, plane_only, Cch, plane);
        uint32_t pos = k - 1u - (uint32_t)(b % k);
        out[x] = (uint8_t)((out[x] & ~(1u << pos)) | ((uint32_t)bit << pos));
    }
    return OR_OK;
}

/* Stream bit b read back from a stego. */
static uint32_t streamk_bit(const uint8_t *st, uint64_t b, uint32_t k, int plane_only,
                            uint32_t Cch, uint32_t plane)
{
    uint64_t x = carrying_index(b / k, plane_only, Cch, plane);
    uint32_t pos = k - 1u - (uint32_t)(b % k);
    return (st[x] >> pos) & 1u;
}

int oracle_streamk_extract(const uint8_t *st, uint64_t C, uint32_t k, int plane_only,
                           uint32_t W, uint32_t H, uint32_t Cch, uint32_t plane, uint8_t *msg,
                           uint64_t cap, int header, uint64_t raw_len, uint64_t *out_len)
{
    uint64_t avail_bits, len, first, s;
    int i;
    if (out_len)
        *out_len = 0;
    if (!streamk_args_ok(C, k, plane_only, W, H, Cch, plane))
        return OR_E_INVAL;
    if (C > 0 && st == 0)
        return OR_E_INVAL;
    avail_bits = (uint64_t)k * carrying_bytes(C, plane_only, W, H);
    if (header) {
        uint64_t nbits = 0, b;
        if (avail_bits < 32u)
            return OR_E_BAD_HEADER;
        for (b = 0; b < 32u; ++b)
            nbits |= (uint64_t)streamk_bit(st, b, k, plane_only, Cch, plane) << (31u - (uint32_t)b);
        if (nbits % 8u != 0u)
            return OR_E_BAD_HEADER;
        if (32u + nbits > avail_bits)
            return OR_E_BAD_HEADER;
        len = nbits / 8u;
        if (len > cap)
            return OR_E_MSG_TOO_SMALL;
        first = 32u;
    } else {
        len = raw_len;
        if (8u * len > avail_bits)
            return OR_E_CAPACITY;
        if (len > cap)
            return OR_E_MSG_TOO_SMALL;
        first = 0u;
    }
    if (len > 0 && msg == 0)
        return OR_E_INVAL;
    for (s = 0; s < len; ++s) {
        uint8_t v = 0;
        for (i = 0; i < 8; ++i)
            v = (uint8_t)(v | (streamk_bit(st, first + 8u * s + (uint64_t)i, k, plane_only, Cch,
                                           plane)
                               << (7 - i)));
        msg[s] = v;
    }
    if (out_len)
        *out_len = len;
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* paper2: Sections VI and VII as printed                                    */
/* ------------------------------------------------------------------------ */

/* Step 7c: the mask applied to data byte y in block i (the fourth mask is
 * printed garbled; by the pattern of the other three it is 1100 0000). */
static uint8_t paper_mask(int i)
{
    switch (i) {
    case 0: return 0x03u; /* 0000 0011 */
    case 1: return 0x0Cu; /* 0000 1100 */
    case 2: return 0x30u; /* 0011 0000 */
    default: return 0xC0u; /* 1100 0000 */
    }
}

static int paper_geom_ok(uint32_t W, uint32_t H, uint32_t Cch, uint32_t plane)
{
    (void)W;
    (void)H;
    return Cch > 0u && plane < Cch;
}

/* Capacity in message bytes: floor(W/4) bytes per row (step 5: size(B)*4 <=
 * size(A)), over all H rows. */
uint64_t oracle_paper2_capacity(uint32_t W, uint32_t H)
{
    return (uint64_t)(W / 4u) * (uint64_t)H;
}

/* Section VI.  The cover is H rows of W pixels with Cch interleaved channels;
 * A is plane `plane` of one row.  N message bytes are divided greedily among
 * the rows (row r takes L = min(N_remaining, floor(W/4)) bytes), and for each
 * block i (0..3) and thread j (0..L-1):
 *   y = (B[j] AND mask_i) >> 2i ;  A[L*i + j] = (A[L*i + j] AND 1111 1100) OR y.
 * out may equal cover.  On error nothing is written. */
int oracle_paper2_embed(const uint8_t *cover, uint8_t *out, uint32_t W,
                        uint32_t H, uint32_t Cch, uint32_t plane,
                        const uint8_t *msg, uint64_t N)
{
    uint64_t C = (uint64_t)W * H * Cch;
    uint64_t Q = W / 4u, rem = N, off = 0;
    uint32_t r;
    if (!paper_geom_ok(W, H, Cch, plane))
        return OR_E_INVAL;
    if (C > 0 && (cover == 0 || out == 0))
        return OR_E_INVAL;
    if (N > 0 && msg == 0)
        return OR_E_INVAL;
    if (N > oracle_paper2_capacity(W, H))
        return OR_E_CAPACITY;

    if (out != cover)
        memcpy(out, cover, (size_t)C);

    for (r = 0; r < H && rem > 0; ++r) {
        uint64_t L = rem < Q ? rem : Q;
        int i;
        uint64_t j;
        for (i = 0; i < 4; ++i) {
            for (j = 0; j < L; ++j) {
                uint64_t x = ((uint64_t)r * W + L * (uint64_t)i + j) * Cch + plane;
                uint8_t y = msg[off + j];
                y = (uint8_t)(y & paper_mask(i));
                y = (uint8_t)(y >> (2 * i));
                out[x] = (uint8_t)((cover[x] & 0xFCu) | y);
            }
        }
        off += L;
        rem -= L;
    }
    return OR_OK;
}

/* Section VII.  Same traversal as the embedding; B is zero-initialised per
 * row (step 4) and for each block i and thread j:
 *   y = (A[L*i + j] AND 0000 0011) << 2i ;  B[j] = B[j] OR y. */
int oracle_paper2_extract(const uint8_t *st, uint32_t W, uint32_t H,
                          uint32_t Cch, uint32_t plane, uint8_t *msg,
                          uint64_t cap, uint64_t N)
{
    uint64_t Q = W / 4u, rem = N, off = 0;
    uint32_t r;
    if (!paper_geom_ok(W, H, Cch, plane))
        return OR_E_INVAL;
    if ((uint64_t)W * H * Cch > 0 && st == 0)
        return OR_E_INVAL;
    if (N > oracle_paper2_capacity(W, H))
        return OR_E_CAPACITY;
    if (N > cap)
        return OR_E_MSG_TOO_SMALL;
    if (N > 0 && msg == 0)
        return OR_E_INVAL;

    for (r = 0; r < H && rem > 0; ++r) {
        uint64_t L = rem < Q ? rem : Q;
        int i;
        uint64_t j;
        for (j = 0; j < L; ++j)
            msg[off + j] = 0;
        for (i = 0; i < 4; ++i) {
            for (j = 0; j < L; ++j) {
                uint64_t x = ((uint64_t)r * W + L * (uint64_t)i + j) * Cch + plane;
                uint8_t y = (uint8_t)(st[x] & 0x03u);
                y = (uint8_t)(y << (2 * i));
                msg[off + j] = (uint8_t)(msg[off + j] | y);
            }
        }
        off += L;
        rem -= L;
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Changed bytes and squared error (Section VIII reports PSNR)               */
/* ------------------------------------------------------------------------ */

/* changed = number of positions where a and b differ;
 * sse = sum of (a[k] - b[k])^2.  MSE = sse / n, PSNR = 10 log10(255^2 / MSE). */
void oracle_changed_bytes(const uint8_t *a, const uint8_t *b, uint64_t n,
                          uint64_t *changed, uint64_t *sse)
{
    uint64_t k, c = 0, s = 0;
    for (k = 0; k < n; ++k) {
        int64_t d = (int64_t)a[k] - (int64_t)b[k];
        if (d != 0)
            c += 1u;
        s += (uint64_t)(d * d);
    }
    *changed = c;
    *sse = s;
}
