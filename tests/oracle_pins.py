"""Pins for the CPU oracle: checks against things other than the oracle itself.

Each pin is a plain function taking an ``oracle.Oracle`` handle and raising
``AssertionError`` on a mismatch.  ``test_oracle_pins.py`` runs them against
the committed oracle; ``test_oracle_mutants.py`` runs them against copies of
the oracle with planted mistakes and requires that some pin fails for each.

What pins what:
  * golden fixtures -- hand-worked examples derived from Sections VI/VII and
    the stream convention (tests/golden/*.txt, each citing its source);
  * exhaustive single-byte tables -- every (cover byte, bit) and (cover byte,
    bit pair) against the substitution rule;
  * brute force -- an independent pure-Python bit-list formulation on covers
    of at most 64 bytes, and a per-message-byte formulation of the paper's row
    division;
  * invariants -- round trip, non-LSB bits unchanged, bytes past the message
    untouched, |stego - cover| <= 1 (<= 3 for two bits), sse == changed;
  * the Section VIII session shape (a 1024-byte row carrying a 7x8 secret
    flattened column-major), the Section VIII PSNR gap, and the absolute
    PSNR scale from its definition on hand-worked (sse, n) pairs.
"""
from __future__ import annotations

import math
import os

import numpy as np

import oracle as orc

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


# --------------------------------------------------------------------------
# independent formulations (pure Python, small inputs only)
# --------------------------------------------------------------------------

def brute_stream_bits(msg: bytes, header: bool) -> list[int]:
    s = ((8 * len(msg)).to_bytes(4, "big") + bytes(msg)) if header else bytes(msg)
    return [int(ch) for b in s for ch in format(b, "08b")]


def brute_stream1_embed(cover: bytes, msg: bytes, header: bool):
    bits = brute_stream_bits(msg, header)
    if len(bits) > len(cover):
        return None
    out = list(cover)
    for k, bit in enumerate(bits):
        out[k] = (out[k] - (out[k] % 2)) + bit
    return bytes(out)


def brute_stream1_extract(stego: bytes, cap: int, header: bool, raw_len: int = 0):
    lsb = [b % 2 for b in stego]
    if header:
        if len(stego) < 32:
            return orc.E_BAD_HEADER, b""
        nbits = int("".join(str(b) for b in lsb[:32]), 2)
        if nbits % 8 or 32 + nbits > len(stego):
            return orc.E_BAD_HEADER, b""
        n, base = nbits // 8, 32
        if n > cap:
            return orc.E_MSG_TOO_SMALL, b""
    else:
        n, base = raw_len, 0
        if 8 * n > len(stego):
            return orc.E_CAPACITY, b""
        if n > cap:
            return orc.E_MSG_TOO_SMALL, b""
    out = bytes(int("".join(str(b) for b in lsb[base + 8 * s: base + 8 * s + 8]), 2)
                for s in range(n))
    return orc.OK, out


def brute_paper2_positions(W: int, H: int, Cch: int, plane: int, N: int):
    """For each message byte o, the four (byte index, pair index) it writes,
    derived per byte: row r = o // Q, column j = o % Q, L_r = min(Q, N - r*Q),
    pair i lands at pixel r*W + L_r*i + j of the plane."""
    Q = W // 4
    pos = []
    for o in range(N):
        r, j = divmod(o, Q)
        L = min(Q, N - r * Q)
        pos.append([((r * W + L * i + j) * Cch + plane, i) for i in range(4)])
    return pos


def brute_paper2_embed(cover: bytes, W, H, Cch, plane, msg: bytes):
    Q = W // 4
    if len(msg) > Q * H:
        return None
    out = list(cover)
    for o, places in enumerate(brute_paper2_positions(W, H, Cch, plane, len(msg))):
        pairs = format(msg[o], "08b")  # MSB first: pair 3 is chars 0..1
        for x, i in places:
            p = int(pairs[6 - 2 * i: 8 - 2 * i], 2)
            out[x] = out[x] - (out[x] % 4) + p
    return bytes(out)


def brute_paper2_extract(stego: bytes, W, H, Cch, plane, N):
    msg = []
    for places in brute_paper2_positions(W, H, Cch, plane, N):
        s = ["00"] * 4
        for x, i in places:
            s[3 - i] = format(stego[x] % 4, "02b")
        msg.append(int("".join(s), 2))
    return bytes(msg)


def rng(seed):
    return np.random.default_rng(seed)


# --------------------------------------------------------------------------
# golden fixtures
# --------------------------------------------------------------------------

def load_golden(name: str) -> dict:
    d = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split(":", 1)
            v = v.strip()
            if k in ("cover", "msg", "stego"):
                d[k] = np.array([int(t, 16) for t in v.split()], dtype=np.uint8)
            elif k == "layout":
                d[k] = v
            else:
                d[k] = int(v)
    return d


def golden_names():
    return sorted(n for n in os.listdir(GOLDEN) if n.endswith(".txt"))


def check_golden(o: orc.Oracle, name: str):
    g = load_golden(name)
    lay = g["layout"]
    if lay == "stream1":
        st, out = o.stream1_embed(g["cover"], g["msg"], header=bool(g["header"]))
        assert st == g["status"], (name, st)
        if st == orc.OK:
            assert out.tolist() == g["stego"].tolist(), (name, out)
            ch, sse = o.changed_bytes(g["cover"], out)
            assert (ch, sse) == (g["changed"], g["sse"]), (name, ch, sse)
            st2, m = o.stream1_extract(out, cap=len(g["msg"]), header=bool(g["header"]),
                                       raw_len=len(g["msg"]))
            assert st2 == orc.OK and m.tolist() == g["msg"].tolist(), name
    elif lay == "stream1-extract":
        st, m = o.stream1_extract(g["stego"], cap=64, header=bool(g["header"]))
        assert st == g["status"], (name, st)
    elif lay == "streamk":
        geom = (g["width"], g["height"], g["channels"], g["plane"]) if "width" in g else None
        sentinel = np.full_like(g["cover"], 0x5A)
        st, out = o.streamk_embed(g["cover"], g["msg"], g["k"], header=bool(g["header"]),
                                  geom=geom, out=sentinel.copy())
        assert st == g["status"], (name, st)
        if st != orc.OK:
            assert out.tolist() == sentinel.tolist()
            return
        assert out.tolist() == g["stego"].tolist(), (name, out)
        st2, m = o.streamk_extract(out, g["k"], cap=len(g["msg"]), header=bool(g["header"]),
                                   raw_len=len(g["msg"]), geom=geom)
        assert st2 == orc.OK and m.tolist() == g["msg"].tolist(), name
    elif lay == "paper2":
        W, H, C, p = g["width"], g["height"], g["channels"], g["plane"]
        sentinel = np.full_like(g["cover"], 0x5A)
        st, out = o.paper2_embed(g["cover"], W, H, C, p, g["msg"], out=sentinel.copy())
        assert st == g["status"], (name, st)
        if st != orc.OK:
            assert out.tolist() == sentinel.tolist(), "nothing written on error"
            return
        assert out.tolist() == g["stego"].tolist(), (name, out)
        if "changed" in g:
            assert o.changed_bytes(g["cover"], out) == (g["changed"], g["sse"]), name
        st2, m = o.paper2_extract(out, W, H, C, p, len(g["msg"]))
        assert st2 == orc.OK and m.tolist() == g["msg"].tolist(), name
    else:
        raise AssertionError("unknown layout " + lay)


def pin_golden(o):
    for n in golden_names():
        check_golden(o, n)


# --------------------------------------------------------------------------
# exhaustive single-byte tables
# --------------------------------------------------------------------------

def pin_table_stream1(o):
    """Every cover byte value with every bit: (c & ~1) | bit, raw stream."""
    for c in range(256):
        cover = np.full(8, c, np.uint8)
        for bit in (0, 1):
            msg = np.array([0xFF if bit else 0x00], np.uint8)
            st, out = o.stream1_embed(cover, msg, header=False)
            assert st == orc.OK
            want = (c - c % 2) + bit
            assert out.tolist() == [want] * 8, (c, bit, out)


def pin_table_paper2(o):
    """Every cover byte value with every bit pair: (c & ~3) | pair.  A data
    byte p*0x55 has pair p in all four positions; one row of W = 4 holds it."""
    for c in range(256):
        cover = np.full(4, c, np.uint8)
        for p in range(4):
            msg = np.array([p * 0x55], np.uint8)
            st, out = o.paper2_embed(cover, 4, 1, 1, 0, msg)
            assert st == orc.OK
            want = (c - c % 4) + p
            assert out.tolist() == [want] * 4, (c, p, out)


# --------------------------------------------------------------------------
# brute force on tiny covers
# --------------------------------------------------------------------------

def pin_brute_stream1(o):
    r = rng(11)
    for C in range(0, 65):
        cover = r.integers(0, 256, C, dtype=np.uint8)
        for header in (False, True):
            cap = C // 8 - (4 if header else 0)
            for m in sorted({0, 1, max(cap, 0), max(cap // 2, 0), max(cap + 1, 0)}):
                msg = r.integers(0, 256, m, dtype=np.uint8)
                want = brute_stream1_embed(bytes(cover), bytes(msg), header)
                st, out = o.stream1_embed(cover, msg, header=header)
                if want is None:
                    assert st == orc.E_CAPACITY, (C, m, header, st)
                    continue
                assert st == orc.OK, (C, m, header, st)
                assert bytes(out) == want, (C, m, header)
                for cap_x in (m, m + 3, max(m - 1, 0)):
                    bst, bmsg = brute_stream1_extract(want, cap_x, header, raw_len=m)
                    ost, omsg = o.stream1_extract(out, cap=cap_x, header=header, raw_len=m)
                    assert ost == bst, (C, m, cap_x, ost, bst)
                    if ost == orc.OK:
                        assert bytes(omsg) == bmsg
    # extraction of arbitrary (mostly invalid) headers
    for t in range(400):
        C = int(r.integers(0, 80))
        st_bytes = r.integers(0, 256, C, dtype=np.uint8)
        if C >= 32 and t % 2:
            # plant a valid-looking small header
            n = int(r.integers(0, max((C - 32) // 8, 0) + 2))
            hdr = format(8 * n, "032b")
            for k in range(32):
                st_bytes[k] = (st_bytes[k] & 0xFE) | int(hdr[k])
        cap = int(r.integers(0, 8))
        bst, bmsg = brute_stream1_extract(bytes(st_bytes), cap, True)
        ost, omsg = o.stream1_extract(st_bytes, cap=cap, header=True)
        assert ost == bst, (C, cap, ost, bst)
        assert bytes(omsg) == bmsg


def pin_brute_paper2(o):
    r = rng(12)
    for W in (4, 5, 7, 8, 9, 12, 16, 21):
        for H in (1, 2, 3):
            for Cch in (1, 3, 4):
                for plane in range(Cch):
                    cap = (W // 4) * H
                    cover = r.integers(0, 256, W * H * Cch, dtype=np.uint8)
                    for N in sorted({0, 1, cap // 2, cap, cap + 1}):
                        msg = r.integers(0, 256, N, dtype=np.uint8)
                        want = brute_paper2_embed(bytes(cover), W, H, Cch, plane, bytes(msg))
                        st, out = o.paper2_embed(cover, W, H, Cch, plane, msg)
                        if want is None:
                            assert st == orc.E_CAPACITY
                            continue
                        assert st == orc.OK
                        assert bytes(out) == want, (W, H, Cch, plane, N)
                        st2, m2 = o.paper2_extract(out, W, H, Cch, plane, N)
                        assert st2 == orc.OK
                        assert bytes(m2) == brute_paper2_extract(want, W, H, Cch, plane, N)
                        assert bytes(m2) == bytes(msg)


# --------------------------------------------------------------------------
# invariants on random covers
# --------------------------------------------------------------------------

def pin_invariants_stream1(o):
    r = rng(13)
    for C in (32, 33, 100, 255, 256, 1000, 4096, 10007):
        cover = r.integers(0, 256, C, dtype=np.uint8)
        for header in (True, False):
            cap = C // 8 - (4 if header else 0)
            for m in sorted({0, 1, cap // 3, cap}):
                if m < 0 or m > cap:
                    continue
                msg = r.integers(0, 256, m, dtype=np.uint8)
                st, out = o.stream1_embed(cover, msg, header=header)
                assert st == orc.OK
                T = 8 * (m + (4 if header else 0))
                d = out.astype(np.int16) - cover.astype(np.int16)
                assert np.all(np.abs(d) <= 1)
                assert np.all(((out ^ cover) & 0xFE) == 0)
                assert np.array_equal(out[T:], cover[T:])
                ch, sse = o.changed_bytes(cover, out)
                assert ch == sse == int(np.count_nonzero(d))
                st2, m2 = o.stream1_extract(out, cap=m, header=header, raw_len=m)
                assert st2 == orc.OK and np.array_equal(m2, msg)
                # in place gives the same bytes
                buf = cover.copy()
                st3, buf = o.stream1_embed_inplace(buf, msg, header=header)
                assert st3 == orc.OK and np.array_equal(buf, out)


def pin_invariants_paper2(o):
    r = rng(14)
    for (W, H, Cch) in ((64, 8, 1), (65, 7, 3), (100, 5, 4), (1024, 1, 1)):
        cover = r.integers(0, 256, W * H * Cch, dtype=np.uint8)
        cap = (W // 4) * H
        for plane in range(Cch):
            for N in (0, 1, cap // 2 + 1, cap):
                msg = r.integers(0, 256, N, dtype=np.uint8)
                st, out = o.paper2_embed(cover, W, H, Cch, plane, msg)
                assert st == orc.OK
                d = out.astype(np.int16) - cover.astype(np.int16)
                assert np.all(np.abs(d) <= 3)
                assert np.all(((out ^ cover) & 0xFC) == 0)
                touched = np.zeros(cover.size, bool)
                for places in brute_paper2_positions(W, H, Cch, plane, N):
                    for x, _ in places:
                        touched[x] = True
                assert np.array_equal(out[~touched], cover[~touched])
                assert int(touched.sum()) == 4 * N
                st2, m2 = o.paper2_extract(out, W, H, Cch, plane, N)
                assert st2 == orc.OK and np.array_equal(m2, msg)


def pin_statistics(o):
    """A uniform random message flips a carried LSB with probability 1/2
    (one bit) and changes a carried byte with probability 3/4 (two bits)."""
    r = rng(15)
    C = 1 << 16
    cover = r.integers(0, 256, C, dtype=np.uint8)
    m = C // 8 - 4
    msg = r.integers(0, 256, m, dtype=np.uint8)
    st, out = o.stream1_embed(cover, msg, header=True)
    ch, _ = o.changed_bytes(cover, out)
    T = 8 * (m + 4)
    sigma = math.sqrt(T * 0.25)
    assert abs(ch - T / 2) < 6 * sigma, ch
    W, H = 256, 64
    cov2 = r.integers(0, 256, W * H, dtype=np.uint8)
    N = (W // 4) * H
    st, out2 = o.paper2_embed(cov2, W, H, 1, 0, r.integers(0, 256, N, dtype=np.uint8))
    ch2, _ = o.changed_bytes(cov2, out2)
    n2 = 4 * N
    assert abs(ch2 - 0.75 * n2) < 6 * math.sqrt(n2 * 0.75 * 0.25), ch2


# --------------------------------------------------------------------------
# errors
# --------------------------------------------------------------------------

def pin_errors(o):
    r = rng(16)
    cover = r.integers(0, 256, 64, dtype=np.uint8)
    sentinel = np.full(64, 0x77, np.uint8)
    # capacity: 64 bytes carry 8 stream bytes = 4 message bytes behind a header
    st, out = o.stream1_embed(cover, np.zeros(5, np.uint8), header=True, out=sentinel.copy())
    assert st == orc.E_CAPACITY and np.array_equal(out, sentinel)
    st, out = o.stream1_embed(cover, np.zeros(4, np.uint8), header=True, out=sentinel.copy())
    assert st == orc.OK
    st, out = o.stream1_embed(cover, np.zeros(9, np.uint8), header=False, out=sentinel.copy())
    assert st == orc.E_CAPACITY and np.array_equal(out, sentinel)
    # header shorter than 32 bytes
    st, _ = o.stream1_extract(cover[:31], cap=100, header=True)
    assert st == orc.E_BAD_HEADER
    # 9 or 31 bits fit in 64 bytes but are not whole bytes; 40 bits need
    # 72 bytes > 64
    for nbits, want in ((9, orc.E_BAD_HEADER), (31, orc.E_BAD_HEADER),
                        (40, orc.E_BAD_HEADER), (32, orc.OK), (0, orc.OK)):
        c = cover.copy()
        h = format(nbits, "032b")
        for k in range(32):
            c[k] = (c[k] & 0xFE) | int(h[k])
        st, m = o.stream1_extract(c, cap=100, header=True)
        assert st == want, (nbits, st)
        if st == orc.OK:
            assert m.size == nbits // 8
    # message buffer too small for a valid header
    c = cover.copy()
    h = format(32, "032b")
    for k in range(32):
        c[k] = (c[k] & 0xFE) | int(h[k])
    st, _ = o.stream1_extract(c, cap=3, header=True)
    assert st == orc.E_MSG_TOO_SMALL
    st, _ = o.stream1_extract(c, cap=4, header=True)
    assert st == orc.OK
    # raw extraction bounds
    st, _ = o.stream1_extract(cover, cap=100, header=False, raw_len=9)
    assert st == orc.E_CAPACITY
    st, _ = o.stream1_extract(cover, cap=2, header=False, raw_len=3)
    assert st == orc.E_MSG_TOO_SMALL
    # paper2 geometry and capacity
    st, _ = o.paper2_embed(cover, 8, 8, 1, 1, np.zeros(1, np.uint8))
    assert st == orc.E_INVAL  # plane >= channels
    st, _ = o.paper2_embed(cover[:12], 3, 4, 1, 0, np.zeros(1, np.uint8))
    assert st == orc.E_CAPACITY  # floor(3/4) = 0 bytes per row
    st, _ = o.paper2_extract(cover, 8, 8, 1, 0, 17)
    assert st == orc.E_CAPACITY
    st, _ = o.paper2_extract(cover, 8, 8, 1, 0, 5, cap=4)
    assert st == orc.E_MSG_TOO_SMALL


# --------------------------------------------------------------------------
# Section VIII
# --------------------------------------------------------------------------

def pin_section8_session(o):
    """Section VIII: a 1024x1 image row D carries a 7x8 secret A sent as
    A(1:56) (column-major); extract(E, 56) then reshaping 7x8 column-major
    gives A back.  Pair i of byte j sits at A[56*i + j]; bytes 224.. untouched."""
    r = rng(17)
    D = r.integers(0, 256, 1024, dtype=np.uint8)
    A = r.integers(0, 256, (7, 8), dtype=np.uint8)
    B = A.ravel(order="F")
    assert B.size == 56
    st, E = o.paper2_embed(D, 1024, 1, 1, 0, B)
    assert st == orc.OK
    for j in range(56):
        for i in range(4):
            assert E[56 * i + j] & 3 == (int(B[j]) >> (2 * i)) & 3
            assert E[56 * i + j] >> 2 == D[56 * i + j] >> 2
    assert np.array_equal(E[224:], D[224:])
    st, F = o.paper2_extract(E, 1024, 1, 1, 0, 56)
    assert st == orc.OK
    G = F.reshape((7, 8), order="F")
    assert np.array_equal(G, A)


def pin_psnr_gap(o):
    """Section VIII prints PSNR 51.6715 for an 8-bit cover and 56.4427 for a
    24-bit cover carrying the same 7x8 secret.  With MSE averaged over every
    cover byte (all channels), embedding in one plane of a 3-channel cover
    leaves the squared error unchanged and triples the byte count, so the gap
    is exactly 10*log10(3) = 4.77121 dB, which is the printed gap to the
    printed precision."""
    assert abs((56.4427 - 51.6715) - 10 * math.log10(3)) < 1.5e-4
    r = rng(18)
    H, W = 32, 1024
    rgb = r.integers(0, 256, (H, W, 3), dtype=np.uint8)
    gray = np.ascontiguousarray(rgb[:, :, 0])
    secret = r.integers(0, 256, 56, dtype=np.uint8)
    st, s3 = o.paper2_embed(rgb, W, H, 3, 0, secret)
    assert st == orc.OK
    st, s1 = o.paper2_embed(gray, W, H, 1, 0, secret)
    assert st == orc.OK
    _, sse3 = o.changed_bytes(rgb, s3)
    _, sse1 = o.changed_bytes(gray, s1)
    assert sse3 == sse1 > 0
    gap = o.psnr(sse3, rgb.size) - o.psnr(sse1, gray.size)
    assert abs(gap - 10 * math.log10(3)) < 1e-9
    # planes 1 and 2 of the stego are the cover's
    assert np.array_equal(s3.reshape(H, W, 3)[:, :, 1:], rgb[:, :, 1:])


def pin_psnr_value(o):
    """The absolute scale of the Section VIII measure, fixed by its
    definition PSNR = 10 log10(255^2 / MSE), MSE = sse / n, values worked by
    hand (the gap pin above is blind to the peak, which cancels):
      * sse = 1 over n = 1 byte: MSE 1, so 10 log10(65025) = 20 log10(255)
        = 48.1308036 dB (log10 255 = 2.40654018);
      * sse = n (every byte off by one): the same 48.1308 dB for any n;
      * sse = 650250 over n = 1000: MSE 650.25 = 65025 / 100, so 20 dB;
      * sse = 65025 over n = 1: MSE = peak^2, so 0 dB;
      * sse = 0: no distortion, infinite PSNR."""
    assert abs(o.psnr(1, 1) - 48.1308036086791) < 1e-9
    assert abs(o.psnr(786432, 786432) - 48.1308036086791) < 1e-9
    assert abs(o.psnr(650250, 1000) - 20.0) < 1e-9
    assert abs(o.psnr(65025, 1) - 0.0) < 1e-9
    assert o.psnr(0, 12345) == math.inf
    # halving the error adds 10 log10 2 dB, whatever the scale
    assert abs(o.psnr(2, 1000) - o.psnr(4, 1000) - 10 * math.log10(2)) < 1e-9


def pin_changed_definition(o):
    """changed = #{k: a[k] != b[k]}, sse = sum (a[k]-b[k])^2, checked against
    numpy on arbitrary (not only LSB-differing) byte arrays."""
    r = rng(19)
    for n in (0, 1, 7, 1000):
        a = r.integers(0, 256, n, dtype=np.uint8)
        b = a.copy()
        idx = r.integers(0, max(n, 1), n // 3) if n else np.zeros(0, np.int64)
        b[idx] = r.integers(0, 256, idx.size, dtype=np.uint8)
        d = a.astype(np.int64) - b.astype(np.int64)
        assert o.changed_bytes(a, b) == (int(np.count_nonzero(d)), int((d * d).sum()))
    a = np.zeros(4, np.uint8)
    b = np.array([255, 0, 1, 0], np.uint8)
    assert o.changed_bytes(a, b) == (2, 255 * 255 + 1)


# --------------------------------------------------------------------------
# k bits per carrying byte, all bytes or one plane
# --------------------------------------------------------------------------

def brute_streamk_embed(cover: bytes, msg: bytes, k: int, header: bool, geom=None):
    bits = brute_stream_bits(msg, header)
    if geom is None:
        carry = list(range(len(cover)))
    else:
        W, H, C, p = geom
        carry = [x * C + p for x in range(W * H)]
    if -(-len(bits) // k) > len(carry):
        return None
    out = list(cover)
    for x in range(0, len(bits), k):
        field = bits[x:x + k]
        pos = carry[x // k]
        value = format(out[pos], "08b")           # bit 7 first
        lo = list(value[8 - k:])                  # the k low bits, high first
        lo[:len(field)] = [str(b) for b in field]
        out[pos] = int(value[:8 - k] + "".join(lo), 2)
    return bytes(out)


def pin_golden_streamk_relation(o):
    """k = 1 over all bytes is the one-bit stream layout."""
    r = rng(21)
    for C in (0, 40, 333, 4096):
        cover = r.integers(0, 256, C, dtype=np.uint8)
        for header in (True, False):
            cap = max(C // 8 - (4 if header else 0), 0)
            msg = r.integers(0, 256, cap, dtype=np.uint8)
            a = o.stream1_embed(cover, msg, header=header)
            b = o.streamk_embed(cover, msg, 1, header=header)
            assert a[0] == b[0] and np.array_equal(a[1], b[1]), (C, header)


def pin_table_streamk(o):
    """Every cover byte value with every k-bit field, k = 2, 3, 4: eight
    carrying bytes all get (c & ~(2^k - 1)) | f."""
    for k in (2, 3, 4):
        for f in range(1 << k):
            bits = format(f, "0%db" % k) * 8       # eight fields
            msg = np.array([int(bits[i:i + 8], 2) for i in range(0, 8 * k, 8)], np.uint8)
            for c in range(256):
                st, out = o.streamk_embed(np.full(8, c, np.uint8), msg, k, header=False)
                assert st == orc.OK
                want = (c - c % (1 << k)) + f
                assert out.tolist() == [want] * 8, (k, f, c, out)


def pin_brute_streamk(o):
    r = rng(22)
    for k in (1, 2, 3, 4):
        for geom in (None, (3, 2, 3, 1), (5, 3, 1, 0), (4, 4, 4, 3), (2, 5, 2, 0)):
            for C in ((0, 7, 31, 40, 64) if geom is None else (geom[0] * geom[1] * geom[2],)):
                cover = r.integers(0, 256, C, dtype=np.uint8)
                ncarry = C if geom is None else geom[0] * geom[1]
                for header in (False, True):
                    cap = max(k * ncarry // 8 - (4 if header else 0), 0)
                    for m in sorted({0, 1, cap // 2, cap, cap + 1}):
                        msg = r.integers(0, 256, m, dtype=np.uint8)
                        want = brute_streamk_embed(bytes(cover), bytes(msg), k, header, geom)
                        st, out = o.streamk_embed(cover, msg, k, header=header, geom=geom)
                        if want is None:
                            assert st == orc.E_CAPACITY, (k, geom, C, m, header, st)
                            continue
                        assert st == orc.OK and bytes(out) == want, (k, geom, C, m, header)
                        st2, m2 = o.streamk_extract(out, k, cap=m, header=header, raw_len=m,
                                                    geom=geom)
                        assert st2 == orc.OK and bytes(m2) == bytes(msg), (k, geom, C, m)


def pin_invariants_streamk(o):
    r = rng(23)
    for k in (2, 3, 4):
        for geom in (None, (64, 9, 3, 2), (33, 7, 4, 0)):
            C = 5000 if geom is None else geom[0] * geom[1] * geom[2]
            cover = r.integers(0, 256, C, dtype=np.uint8)
            ncarry = C if geom is None else geom[0] * geom[1]
            cap = k * ncarry // 8 - 4
            for m in (0, cap // 3, cap):
                msg = r.integers(0, 256, m, dtype=np.uint8)
                st, out = o.streamk_embed(cover, msg, k, header=True, geom=geom)
                assert st == orc.OK
                d = out.astype(np.int16) - cover.astype(np.int16)
                assert np.all(np.abs(d) < (1 << k))
                assert np.all(((out ^ cover) & (0xFF ^ ((1 << k) - 1))) == 0)
                T = -(-8 * (m + 4) // k)  # carrying bytes used
                if geom is None:
                    assert np.array_equal(out[T:], cover[T:])
                else:
                    W, H, Cc, p = geom
                    mask = np.ones(C, bool)
                    mask[np.arange(T) * Cc + p] = False
                    assert np.array_equal(out[mask], cover[mask])
                st2, m2 = o.streamk_extract(out, k, cap=m, header=True, geom=geom)
                assert st2 == orc.OK and np.array_equal(m2, msg)


def pin_errors_streamk(o):
    c = np.zeros(64, np.uint8)
    assert o.streamk_embed(c, np.zeros(1, np.uint8), 0, header=False)[0] == orc.E_INVAL
    assert o.streamk_embed(c, np.zeros(1, np.uint8), 5, header=False)[0] == orc.E_INVAL
    assert o.streamk_embed(c, np.zeros(1, np.uint8), 2, header=False,
                           geom=(8, 8, 1, 1))[0] == orc.E_INVAL          # plane >= channels
    assert o.streamk_embed(c, np.zeros(1, np.uint8), 2, header=False,
                           geom=(8, 4, 3, 0))[0] == orc.E_INVAL          # size mismatch
    # 64 bytes x 3 bits = 192 bits = 24 bytes: 20 message bytes behind the header
    assert o.streamk_embed(c, np.zeros(20, np.uint8), 3, header=True)[0] == orc.OK
    assert o.streamk_embed(c, np.zeros(21, np.uint8), 3, header=True)[0] == orc.E_CAPACITY
    # k = 2: header bits 28..31 sit in carrying bytes 14 and 15; a count of 9
    # bits (fields 2, 1) fits 64 bytes but is not whole bytes; 8 (fields 2, 0)
    # is one message byte
    h9 = np.zeros(64, np.uint8)
    h9[14], h9[15] = 2, 1
    assert o.streamk_extract(h9, 2, cap=8, header=True)[0] == orc.E_BAD_HEADER
    h8 = np.zeros(64, np.uint8)
    h8[14] = 2
    st, m = o.streamk_extract(h8, 2, cap=8, header=True)
    assert st == orc.OK and m.size == 1
    # a header needs 32 stream bits: 10 bytes at k = 3 (30 bits) are too few
    assert o.streamk_extract(np.zeros(10, np.uint8), 3, header=True)[0] == orc.E_BAD_HEADER
    assert o.streamk_extract(np.zeros(11, np.uint8), 3, header=True)[0] == orc.OK


PINS = [
    ("golden", pin_golden),
    ("table_stream1", pin_table_stream1),
    ("table_paper2", pin_table_paper2),
    ("brute_stream1", pin_brute_stream1),
    ("brute_paper2", pin_brute_paper2),
    ("invariants_stream1", pin_invariants_stream1),
    ("invariants_paper2", pin_invariants_paper2),
    ("statistics", pin_statistics),
    ("errors", pin_errors),
    ("section8_session", pin_section8_session),
    ("psnr_gap", pin_psnr_gap),
    ("psnr_value", pin_psnr_value),
    ("changed_definition", pin_changed_definition),
    ("streamk_k1_is_stream1", pin_golden_streamk_relation),
    ("table_streamk", pin_table_streamk),
    ("brute_streamk", pin_brute_streamk),
    ("invariants_streamk", pin_invariants_streamk),
    ("errors_streamk", pin_errors_streamk),
]
