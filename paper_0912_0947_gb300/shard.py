"""Covers over several GPUs, one process per GPU.

A batch: covers are independent, so the batch shards with no exchange on
the data path: ``stego_partition`` gives every cover a rank by byte volume,
each rank runs the batched calls on its own covers, and the per-cover
results are gathered on the host afterwards
(``torch.distributed.all_gather_object``: a few bytes per cover, no device
data).

One cover: in the one-bit stream layout stream byte s is carried by cover
bytes 8s..8s+7 and by nothing else, so a cover also splits at any cover
offset that is a multiple of 8 (of 16 here, which keeps every slice on the
vector path).  A slice's stream bytes are a run of header bytes and a run
of message bytes, each embedded or extracted by a raw (headerless) library
call on the slice; the header's four bytes are known to the embedding ranks
(8m, big-endian), and an extracting rank reads them from the first 32
stego bytes before it cuts its own message bytes.

Marshalling only: the steganography runs in the library's kernels on each
rank.
"""
from __future__ import annotations

import numpy as np
import torch

from . import (E_BAD_HEADER, E_CAPACITY, FUSE_STATS, StegoError, new_result, stego_embed,
               stego_extract, stego_partition)

HEADER_BYTES = 4             # BE32 bit count in front of the message
HEADER_COVER = 8 * HEADER_BYTES


def my_covers(sizes, rank: int, world: int) -> np.ndarray:
    """Indices (ascending) of the covers rank `rank` of `world` processes."""
    rank_of, _ = stego_partition(sizes, world)
    return np.nonzero(rank_of == rank)[0]


def gather_results(mine: np.ndarray, results, n: int, group=None) -> list:
    """Per-cover results of every rank, in cover order.  `mine` are this
    rank's cover indices and `results` its results for them (same order);
    with one process no collective runs."""
    import torch.distributed as dist
    part = list(zip((int(i) for i in mine), results))
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        parts = [None] * dist.get_world_size(group)
        dist.all_gather_object(parts, part, group=group)
    else:
        parts = [part]
    out = [None] * n
    for p in parts:
        for i, r in p:
            out[i] = r
    return out


def run_sharded(sizes, rank: int, world: int, compute, group=None) -> list:
    """compute(indices) -> results for those covers, run on this rank's
    share; returns every cover's result in cover order."""
    mine = my_covers(sizes, rank, world)
    return gather_results(mine, compute(mine), len(sizes), group)


# ---------------------------------------------------------------- one cover


def cover_slices(C: int, world: int) -> list[tuple[int, int]]:
    """Cover byte ranges [c0, c1) of a C-byte cover split among `world`
    ranks: near-equal byte counts, every boundary but the cover's end a
    multiple of 16 (a slice may be empty when C < 16 * world)."""
    if world < 1:
        raise ValueError("world must be at least 1")
    b = [((r * C) // world) & ~15 for r in range(world)] + [C]
    return [(b[r], b[r + 1]) for r in range(world)]


def slice_message_range(c0: int, c1: int, m: int, header: bool = True) -> tuple[int, int]:
    """Message bytes [lo, hi) that cover bytes [c0, c1) carry (c0 a multiple
    of 8) for an m-byte message, behind the header or raw."""
    hb = HEADER_BYTES if header else 0
    T = 8 * (m + hb)                       # cover bytes the stream occupies
    a = max(c0 // 8, hb)                   # first message stream byte here
    se = max(min(c1, T) // 8, a)           # stream bytes end here
    return a - hb, se - hb


def slice_pieces(c0: int, c1: int, m: int, header: bool = True) -> list[tuple]:
    """The raw calls cover bytes [c0, c1) take, in order, as tuples
    (kind, a, b, lo, hi): cover bytes [a, b) carry header bytes [lo, hi)
    (kind "header") or message bytes [lo, hi) (kind "msg", which also
    copies the cover bytes past the stream)."""
    out = []
    h1 = min(c1, HEADER_COVER) if header else 0
    if c0 < h1:
        out.append(("header", c0, h1, c0 // 8, h1 // 8))
    a = max(c0, h1)
    if c1 > a:
        lo, hi = slice_message_range(c0, c1, m, header)
        out.append(("msg", a, c1, lo, hi))
    return out


def header_bytes(m: int) -> bytes:
    """The stream's header: the message's bit count, big-endian."""
    return (8 * m).to_bytes(HEADER_BYTES, "big")


def _check_stream(C: int, m: int, header: bool) -> None:
    hb = HEADER_BYTES if header else 0
    if m < 0 or 8 * (m + hb) > C or (header and 8 * m >= 1 << 32):
        raise StegoError(E_CAPACITY, "stream of %d message bytes in %d cover bytes" % (m, C))


class CoverSlice:
    """Rank-side state of one slice, cover bytes [c0, c1) of a C-byte cover
    carrying an m-byte message: the pieces' plan, the header bytes the
    slice carries (on the device) and one result per piece, all made once
    so that `embed` and `extract` only issue the library calls.  A stream
    that does not fit C bytes raises StegoError(E_CAPACITY) here, before
    anything is launched, on every rank alike."""

    def __init__(self, c0: int, c1: int, C: int, m: int, header: bool = True,
                 device="cuda"):
        if c0 % 16 or not 0 <= c0 <= c1 <= C:
            raise ValueError("a slice starts at a multiple of 16 inside the cover")
        _check_stream(C, m, header)
        self.c0, self.c1, self.C, self.m, self.header = c0, c1, C, m, header
        self.pieces = slice_pieces(c0, c1, m, header)
        self.lo, self.hi = slice_message_range(c0, c1, m, header)
        self.results = new_result(device, n=max(len(self.pieces), 1))
        self.xres = new_result(device)
        self.hdr = None
        for kind, a, b, plo, phi in self.pieces:
            if kind == "header":
                self.hdr = torch.tensor(list(header_bytes(m)[plo:phi]),
                                        dtype=torch.uint8).to(device)

    def embed(self, cover_s, stego_s, msg_part, stream=None) -> None:
        """stego_s <- the slice of the stego (`cover_s`, `stego_s`: the
        slice's c1 - c0 bytes; `stego_s` may be `cover_s`; `msg_part`:
        message bytes [lo, hi))."""
        n = self.c1 - self.c0
        if cover_s.numel() != n or stego_s.numel() != n:
            raise ValueError("slice tensors must hold %d bytes" % n)
        if (0 if msg_part is None else msg_part.numel()) != self.hi - self.lo:
            raise ValueError("msg_part must hold message bytes [%d, %d)" % (self.lo, self.hi))
        # the pieces write disjoint bytes: the message piece goes first, so
        # the header's small launch waits on it instead of delaying it
        for i in reversed(range(len(self.pieces))):
            kind, a, b, plo, phi = self.pieces[i]
            src = self.hdr if kind == "header" else (msg_part if phi > plo else None)
            stego_embed(cover_s[a - self.c0: b - self.c0], stego_s[a - self.c0: b - self.c0],
                        src, FUSE_STATS, self.results[i], stream=stream)

    def stats(self, stream=None) -> tuple[int, int]:
        """(changed, sse) of the last embed (waits for `stream`)."""
        from . import read_result
        _sync(stream, self.results.device)
        rr = read_result(self.results)[: len(self.pieces)]
        return sum(r["changed"] for r in rr), sum(r["sse"] for r in rr)

    def extract(self, stego_s, out_part, stream=None) -> None:
        """out_part[:hi - lo] <- message bytes [lo, hi) from the slice's
        stego bytes (nothing past them is written)."""
        if self.hi == self.lo:
            return
        if out_part is None or out_part.numel() < self.hi - self.lo:
            raise ValueError("out_part must hold %d bytes" % (self.hi - self.lo))
        hb = HEADER_BYTES if self.header else 0
        a = 8 * (self.lo + hb) - self.c0   # first carrying byte in the slice
        stego_extract(stego_s[a: a + 8 * (self.hi - self.lo)], out_part, self.hi - self.lo, 0,
                      self.xres, stream=stream)


def embed_slice(cover_s, stego_s, c0: int, C: int, m: int, msg_part, header: bool = True,
                stream=None) -> CoverSlice:
    """One-off form of CoverSlice(c0, c0 + len(cover_s), C, m).embed(...);
    returns the CoverSlice (its `stats` are the slice's changed/sse)."""
    sl = CoverSlice(c0, c0 + cover_s.numel(), C, m, header, cover_s.device)
    sl.embed(cover_s, stego_s, msg_part, stream)
    return sl


def _sync(stream, device) -> None:
    """Wait for the work the library calls queued on `stream` (a torch
    stream, or None for the device's current stream)."""
    if isinstance(stream, torch.cuda.Stream):
        stream.synchronize()
    else:
        torch.cuda.synchronize(device)


def read_header(stego_head, C: int, cap: int | None = None, stream=None) -> int:
    """Message length m from the first 32 stego bytes of a C-byte cover
    (a device tensor of at least 32 bytes): the library extracts the four
    header bytes, the host applies the header extraction's checks (bit
    count a multiple of 8 and inside the cover; with `cap`, m <= cap) and
    raises StegoError(E_BAD_HEADER / E_MSG_TOO_SMALL) like it."""
    from . import E_MSG_TOO_SMALL
    if C < HEADER_COVER or stego_head.numel() < HEADER_COVER:
        raise StegoError(E_BAD_HEADER, "read_header")
    hb = torch.empty(HEADER_BYTES, dtype=torch.uint8, device=stego_head.device)
    r = new_result(stego_head.device)
    stego_extract(stego_head[:HEADER_COVER], hb, HEADER_BYTES, 0, r, stream=stream)
    _sync(stream, hb.device)
    nbits = int.from_bytes(bytes(hb.cpu().tolist()), "big")
    if nbits % 8 or HEADER_COVER + nbits > C:
        raise StegoError(E_BAD_HEADER, "read_header")
    if cap is not None and nbits // 8 > cap:
        raise StegoError(E_MSG_TOO_SMALL, "read_header")
    return nbits // 8


def extract_slice(stego_s, c0: int, C: int, m: int, out_part, header: bool = True,
                  stream=None) -> None:
    """One-off form of CoverSlice(c0, c0 + len(stego_s), C, m).extract: the
    message bytes that stego bytes [c0, c0 + len(stego_s)) of a C-byte
    cover carry into `out_part`."""
    CoverSlice(c0, c0 + stego_s.numel(), C, m, header, stego_s.device).extract(
        stego_s, out_part, stream)
