"""GPU parity of the paper's own layout (Sections VI/VII: one plane, two
bits per byte, greedy row division, pair i of B[j] at A[L*i + j]) against
the CPU oracle, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
import oracle_pins as P
from gpu_util import Guarded, dev, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    return need_gpu()


@pytest.fixture(scope="module")
def O():
    return oracle.load()


def _check(S, O, cover, W, H, Cch, plane, msg, inplace=False, offs=(0, 0)):
    st_o, want = O.paper2_embed(cover, W, H, Cch, plane, msg)
    flags = S.LAYOUT_PAPER2 | S.FUSE_STATS
    geom = (W, H, Cch, plane)
    gc = Guarded(cover.size, offs[0], cover)
    gm = Guarded(msg.size, 0, msg)
    gs = gc if inplace else Guarded(cover.size, offs[1], 0x5A)
    res = S.new_result()
    if st_o != oracle.OK:
        with pytest.raises(S.StegoError) as e:
            S.stego_embed(gc.view, gs.view, gm.view, flags, res, geom=geom)
        assert e.value.status == st_o
        return None
    S.stego_embed(gc.view, gs.view, gm.view, flags, res, geom=geom)
    got = gs.host()
    assert np.array_equal(got, want), (W, H, Cch, plane, msg.size, inplace)
    assert gs.canaries_intact() and gc.canaries_intact()
    r = S.read_result(res)
    assert r["status"] == 0 and r["msg_bytes"] == msg.size
    assert (r["changed"], r["sse"]) == O.changed_bytes(cover, want)
    # extraction with the out-of-band length N (Section VIII: extract(E, N))
    N = msg.size
    st2, mo = O.paper2_extract(want, W, H, Cch, plane, N)
    assert st2 == oracle.OK
    gx = Guarded(N + 2, 1, 0xEE)
    gst = Guarded(want.size, offs[1], want)
    res2 = S.new_result()
    S.stego_extract(gst.view, gx.view, N, S.LAYOUT_PAPER2, res2, geom=geom)
    out = gx.host()
    assert np.array_equal(out[:N], mo) and np.array_equal(out[:N], msg)
    assert np.all(out[N:] == 0xEE) and gx.canaries_intact()
    assert S.read_result(res2)["status"] == 0
    return want


def test_golden(S, O):
    for name in P.golden_names():
        g = P.load_golden(name)
        if g["layout"] != "paper2":
            continue
        got = _check(S, O, g["cover"], g["width"], g["height"], g["channels"], g["plane"],
                     g["msg"])
        if g["status"] == 0:
            assert got.tolist() == g["stego"].tolist(), name


@pytest.mark.parametrize("W,H,Cch", [(4, 1, 1), (5, 3, 1), (9, 4, 3), (33, 7, 3), (64, 16, 4),
                                     (1024, 1, 1), (1027, 9, 3), (4096, 33, 1),
                                     # rows of whole 16-byte vectors: the one-pass kernel
                                     (16, 5, 3), (32, 7, 4), (48, 3, 1), (80, 9, 3), (4000, 6, 4),
                                     (2736, 11, 3)])
def test_random_geometries(S, O, W, H, Cch):
    rng = np.random.default_rng(W * 131 + H * 7 + Cch)
    cover = rng.integers(0, 256, W * H * Cch, dtype=np.uint8)
    cap = (W // 4) * H
    for plane in sorted({0, Cch - 1}):
        for N in sorted({0, 1, cap // 3, cap - 1, cap, cap + 1}):
            if N < 0:
                continue
            msg = rng.integers(0, 256, N, dtype=np.uint8)
            for inplace in (False, True):
                _check(S, O, cover, W, H, Cch, plane, msg, inplace=inplace)
    msg = rng.integers(0, 256, cap // 2, dtype=np.uint8)
    _check(S, O, cover, W, H, Cch, 0, msg, offs=(3, 5))


def test_section8_session(S, O):
    """A 1024x1 row carrying a 7x8 secret sent column-major (Section VIII)."""
    rng = np.random.default_rng(8)
    D = rng.integers(0, 256, 1024, dtype=np.uint8)
    A = rng.integers(0, 256, (7, 8), dtype=np.uint8)
    E = _check(S, O, D, 1024, 1, 1, 0, A.ravel(order="F"))
    assert np.array_equal(E[224:], D[224:])


def test_geometry_errors(S):
    c = torch.zeros(96, dtype=torch.uint8, device="cuda")
    s = torch.zeros(96, dtype=torch.uint8, device="cuda")
    m = torch.zeros(1, dtype=torch.uint8, device="cuda")
    for geom in ((8, 4, 3, 3), (8, 4, 2, 0), (0, 4, 3, 0)):
        with pytest.raises(S.StegoError) as e:
            S.stego_embed(c, s, m, S.LAYOUT_PAPER2, geom=geom)
        assert e.value.status in (S.E_INVAL, S.E_CAPACITY)
    with pytest.raises(S.StegoError) as e:
        S.stego_embed(c, s, m, S.LAYOUT_PAPER2 | S.HEADER_BE32, geom=(8, 4, 3, 0))
    assert e.value.status == S.E_INVAL


def test_full_size_8192_plane0(S, O):
    """8192x8192x3 cover, plane 0, message at the full floor(W/4)*H capacity
    (16,777,216 bytes): one-pass out of place, in place, extraction, all
    against the oracle over every byte."""
    from paper_0912_0947_gb300 import synth
    W = H = 8192
    C = W * H * 3
    N = (W // 4) * H
    cover = synth.uniform_bytes(C, 0xC0FFEE21, "cuda")
    msg = synth.uniform_bytes(N, 0xC0FFEE22, "cuda")
    geom = (W, H, 3, 0)
    stego = torch.empty_like(cover)
    res = S.new_result()
    S.stego_embed(cover, stego, msg, S.LAYOUT_PAPER2 | S.FUSE_STATS, res, geom=geom)
    c_h, m_h = cover.cpu().numpy(), msg.cpu().numpy()
    st, want = O.paper2_embed(c_h, W, H, 3, 0, m_h)
    assert st == 0
    assert np.array_equal(stego.cpu().numpy(), want)
    r = S.read_result(res)
    assert (r["changed"], r["sse"]) == O.changed_bytes(c_h, want)
    buf = cover.clone()
    S.stego_embed(buf, buf, msg, S.LAYOUT_PAPER2, geom=geom)
    assert torch.equal(buf, stego)
    out = torch.empty(N, dtype=torch.uint8, device="cuda")
    S.stego_extract(stego, out, N, S.LAYOUT_PAPER2, geom=geom)
    assert torch.equal(out, msg)
