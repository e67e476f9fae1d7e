"""GPU parity of the stream layout with k = 1..4 bits per carrying byte and
with one-plane carrying (STEGO_BITS / STEGO_PLANE_ONLY) against the CPU
oracle, byte for byte, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
import oracle_pins as P
from gpu_util import Guarded, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    return need_gpu()


@pytest.fixture(scope="module")
def O():
    return oracle.load()


def _flags(S, k, header, geom):
    return S.BITS(k) | (S.HEADER_BE32 if header else 0) | (S.PLANE_ONLY if geom else 0)


def _check(S, O, cover, msg, k, header, geom=None, offs=(0, 0, 0), inplace=False):
    st_o, want = O.streamk_embed(cover, msg, k, header=header, geom=geom)
    flags = _flags(S, k, header, geom) | S.FUSE_STATS
    gc = Guarded(cover.size, offs[0], cover)
    gm = Guarded(msg.size, offs[2], msg)
    gs = gc if inplace else Guarded(cover.size, offs[1], 0x5A)
    res = S.new_result()
    if st_o != oracle.OK:
        with pytest.raises(S.StegoError) as e:
            S.stego_embed(gc.view, gs.view, gm.view, flags, res, geom=geom)
        assert e.value.status == st_o
        return None
    S.stego_embed(gc.view, gs.view, gm.view, flags, res, geom=geom)
    got = gs.host()
    assert np.array_equal(got, want), (cover.size, msg.size, k, header, geom, offs, inplace)
    assert gs.canaries_intact() and gc.canaries_intact() and gm.canaries_intact()
    r = S.read_result(res)
    assert r["status"] == 0 and r["msg_bytes"] == msg.size
    assert (r["changed"], r["sse"]) == O.changed_bytes(cover, want)
    # extraction into a stale buffer
    m = msg.size
    st2, mo = O.streamk_extract(want, k, cap=m + 2, header=header, raw_len=m, geom=geom)
    assert st2 == oracle.OK and np.array_equal(mo, msg)
    gx = Guarded(m + 2, offs[2], 0xEE)
    gst = Guarded(want.size, offs[1], want)
    res2 = S.new_result()
    S.stego_extract(gst.view, gx.view, m, _flags(S, k, header, geom), res2, geom=geom)
    r2 = S.read_result(res2)
    assert r2["status"] == 0 and r2["msg_bytes"] == m
    out = gx.host()
    assert np.array_equal(out[:m], msg) and np.all(out[m:] == 0xEE) and gx.canaries_intact()
    return want


def test_golden(S, O):
    for name in P.golden_names():
        g = P.load_golden(name)
        if g["layout"] != "streamk":
            continue
        geom = (g["width"], g["height"], g["channels"], g["plane"]) if "width" in g else None
        got = _check(S, O, g["cover"], g["msg"], g["k"], bool(g["header"]), geom)
        assert got.tolist() == g["stego"].tolist(), name


@pytest.mark.parametrize("k", [2, 3, 4])
@pytest.mark.parametrize("C", [0, 5, 16, 17, 20, 31, 100, 4096, 4101, 65536 + 24, (1 << 20) + 7])
def test_all_bytes(S, O, k, C):
    rng = np.random.default_rng(C * 7 + k)
    cover = rng.integers(0, 256, C, dtype=np.uint8)
    for header in (True, False):
        cap = S.stego_capacity(C, S.BITS(k) | (S.HEADER_BE32 if header else 0))
        for m in sorted({0, 1, cap // 3, cap, cap + 1}):
            msg = rng.integers(0, 256, m, dtype=np.uint8)
            for inplace in (False, True):
                _check(S, O, cover, msg, k, header, inplace=inplace)
    msg = rng.integers(0, 256, max(cap // 2, 0), dtype=np.uint8)
    _check(S, O, cover, msg, k, True, offs=(3, 7, 1))


@pytest.mark.parametrize("out_off", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("header", [True, False])
def test_extract_k3_output_alignment(S, O, out_off, header):
    """k = 3 extraction from an aligned stego into outputs at every offset
    mod 4 (word stores by lane pairs, 16-bit halves, bytes), with message
    ends at every position of a 12-byte lane pair and several grid-stride
    rounds."""
    C = 3 * 65536 + 48 + 5   # 12291 units and a ragged tail
    rng = np.random.default_rng(31 + out_off + 8 * header)
    cover = rng.integers(0, 256, C, dtype=np.uint8)
    flags = S.BITS(3) | (S.HEADER_BE32 if header else 0)
    cap = S.stego_capacity(C, flags)
    for m in sorted({0, 1, 2, 7, 8, 13, cap // 2 + 3} | {cap - d for d in range(13)}):
        msg = rng.integers(0, 256, m, dtype=np.uint8)
        st, stego = O.streamk_embed(cover, msg, 3, header=header)
        assert st == oracle.OK
        gst = Guarded(C, 0, stego)
        gx = Guarded(m + 5, out_off, 0xEE)
        res = S.new_result()
        S.stego_extract(gst.view, gx.view, m, flags, res)
        r = S.read_result(res)
        assert r["status"] == 0 and r["msg_bytes"] == m
        out = gx.host()
        assert np.array_equal(out[:m], msg), (m, out_off, header)
        assert np.all(out[m:] == 0xEE) and gx.canaries_intact()


@pytest.mark.parametrize("k", [1, 2, 3, 4])
@pytest.mark.parametrize("geom", [(4, 1, 3, 1), (17, 5, 3, 0), (64, 9, 4, 3), (100, 7, 1, 0),
                                  (33, 33, 2, 1)])
def test_one_plane(S, O, k, geom):
    W, H, Cc, p = geom
    rng = np.random.default_rng(W * H * Cc + p + k)
    cover = rng.integers(0, 256, W * H * Cc, dtype=np.uint8)
    for header in (True, False):
        cap = S.stego_capacity(cover.size, _flags(S, k, header, geom), geom=geom)
        for m in sorted({0, cap // 2, cap, cap + 1}):
            msg = rng.integers(0, 256, m, dtype=np.uint8)
            for inplace in (False, True):
                _check(S, O, cover, msg, k, header, geom=geom, inplace=inplace)


def test_errors(S):
    c = torch.zeros(64, dtype=torch.uint8, device="cuda")
    s = torch.zeros(64, dtype=torch.uint8, device="cuda")
    m = torch.zeros(1, dtype=torch.uint8, device="cuda")
    with pytest.raises(S.StegoError) as e:   # one plane needs a matching geometry
        S.stego_embed(c, s, m, S.PLANE_ONLY, geom=(8, 4, 3, 0))
    assert e.value.status == S.E_INVAL
    with pytest.raises(S.StegoError) as e:   # k-bit flags are for the stream layout
        S.stego_embed(c, s, m, S.LAYOUT_PAPER2 | S.BITS(2), geom=(8, 8, 1, 0))
    assert e.value.status == S.E_INVAL
    # 64 bytes x 3 bits = 24 bytes: 20 message bytes behind the header
    S.stego_embed(c, s, torch.zeros(20, dtype=torch.uint8, device="cuda"),
                  S.BITS(3) | S.HEADER_BE32)
    with pytest.raises(S.StegoError) as e:
        S.stego_embed(c, s, torch.zeros(21, dtype=torch.uint8, device="cuda"),
                      S.BITS(3) | S.HEADER_BE32)
    assert e.value.status == S.E_CAPACITY
    # a stego too short for the header at k = 3 (10 bytes = 30 bits)
    res = S.new_result()
    S.stego_extract(c[:10], torch.zeros(8, dtype=torch.uint8, device="cuda"), 0,
                    S.BITS(3) | S.HEADER_BE32, res)
    assert S.read_result(res)["status"] == S.E_BAD_HEADER


@pytest.mark.parametrize("k", [2, 3, 4])
def test_full_size_8192(S, O, k):
    """The 8192x8192x3 cover at full k-bit capacity, every byte against the
    oracle."""
    from paper_0912_0947_gb300 import synth
    C = 8192 * 8192 * 3
    cover = synth.uniform_bytes(C, 0xC0FFEE31 + k, "cuda")
    m = S.stego_capacity(C, S.BITS(k) | S.HEADER_BE32)
    msg = synth.uniform_bytes(m, 0xC0FFEE41 + k, "cuda")
    stego = torch.empty_like(cover)
    res = S.new_result()
    S.stego_embed(cover, stego, msg, S.BITS(k) | S.HEADER_BE32 | S.FUSE_STATS, res)
    c_h, m_h = cover.cpu().numpy(), msg.cpu().numpy()
    st, want = O.streamk_embed(c_h, m_h, k, header=True)
    assert st == 0 and np.array_equal(stego.cpu().numpy(), want)
    r = S.read_result(res)
    assert (r["changed"], r["sse"]) == O.changed_bytes(c_h, want)
    out = torch.empty(m, dtype=torch.uint8, device="cuda")
    res2 = S.new_result()
    S.stego_extract(stego, out, 0, S.BITS(k) | S.HEADER_BE32, res2)
    assert S.read_result(res2)["msg_bytes"] == m and torch.equal(out, msg)


@pytest.mark.parametrize("k", [1, 2, 3, 4])
@pytest.mark.parametrize("cp", [(3, 0), (3, 1), (3, 2), (4, 0), (4, 1), (4, 2), (4, 3)])
def test_one_plane_units(S, O, k, cp):
    """Every (channels, plane) of the 16-pixel unit kernels over many units
    (and grid-stride iterations) with a ragged tail of 5 pixels."""
    Cc, p = cp
    geom = (129, 37, Cc, p)   # 4773 pixels = 298 units + 5
    rng = np.random.default_rng(1000 * k + 10 * Cc + p)
    cover = rng.integers(0, 256, 129 * 37 * Cc, dtype=np.uint8)
    for header in (True, False):
        cap = S.stego_capacity(cover.size, _flags(S, k, header, geom), geom=geom)
        for m in sorted({cap // 3, cap - 1, cap}):
            msg = rng.integers(0, 256, m, dtype=np.uint8)
            for inplace in (False, True):
                _check(S, O, cover, msg, k, header, geom=geom, inplace=inplace)


@pytest.mark.parametrize("offs", [(3, 7, 1), (0, 16, 2), (5, 5, 0)])
def test_one_plane_misaligned(S, O, offs):
    geom = (64, 9, 3, 1)
    rng = np.random.default_rng(sum(offs))
    cover = rng.integers(0, 256, 64 * 9 * 3, dtype=np.uint8)
    for k in (1, 2, 3):
        cap = S.stego_capacity(cover.size, _flags(S, k, True, geom), geom=geom)
        msg = rng.integers(0, 256, cap // 2, dtype=np.uint8)
        _check(S, O, cover, msg, k, True, geom=geom, offs=offs)


def test_full_size_8192_plane0(S, O):
    """The 8192x8192x3 cover, k = 2 on plane 0 at full capacity (the bench
    leg's workload), every byte against the oracle."""
    from paper_0912_0947_gb300 import synth
    C = 8192 * 8192 * 3
    geom = (8192, 8192, 3, 0)
    flags = S.BITS(2) | S.HEADER_BE32 | S.PLANE_ONLY
    cover = synth.uniform_bytes(C, 0xC0FFEE51, "cuda")
    m = S.stego_capacity(C, flags, geom=geom)
    msg = synth.uniform_bytes(m, 0xC0FFEE52, "cuda")
    stego = torch.empty_like(cover)
    res = S.new_result()
    S.stego_embed(cover, stego, msg, flags | S.FUSE_STATS, res, geom=geom)
    c_h, m_h = cover.cpu().numpy(), msg.cpu().numpy()
    st, want = O.streamk_embed(c_h, m_h, 2, header=True, geom=geom)
    assert st == 0 and np.array_equal(stego.cpu().numpy(), want)
    r = S.read_result(res)
    assert (r["changed"], r["sse"]) == O.changed_bytes(c_h, want)
    out = torch.empty(m, dtype=torch.uint8, device="cuda")
    res2 = S.new_result()
    S.stego_extract(stego, out, 0, flags, res2, geom=geom)
    assert S.read_result(res2)["msg_bytes"] == m and torch.equal(out, msg)
    buf = cover.clone()
    S.stego_embed(buf, buf, msg, flags, geom=geom)
    assert torch.equal(buf, stego)
