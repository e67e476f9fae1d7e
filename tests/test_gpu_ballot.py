"""GPU parity of the ballot-gather extraction (stego_extract_ballot) against
the CPU oracle, byte for byte: sizes with every word-tail length, header and
raw, message buffers at every offset mod 4, bad headers, the full-size
cover, and the flags it refuses."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import Guarded, need_gpu
from paper_0912_0947_gb300 import synth

pytestmark = pytest.mark.gpu

SIZES = [32, 40, 48, 64, 100, 4096, 4097 + 8, 65543, 3 * 16384 * 9 + 8, (1 << 20) + 13]


@pytest.fixture(scope="module")
def S():
    return need_gpu()


@pytest.fixture(scope="module")
def O():
    return oracle.load()


def _check(S, O, stego, m, header, moff=0):
    cap = m + 5
    st_o, want = O.stream1_extract(stego, cap=cap, header=header, raw_len=m)
    assert st_o == oracle.OK
    gs = Guarded(stego.size, 0, stego)
    gm = Guarded(cap, moff, 0xEE)
    res = S.new_result()
    S.stego_extract_ballot(gs.view, gm.view, m, S.HEADER_BE32 if header else 0, res)
    r = S.read_result(res)
    assert r["status"] == 0 and r["msg_bytes"] == want.size
    got = gm.host()
    assert np.array_equal(got[: want.size], want), (stego.size, m, header, moff)
    assert np.all(got[want.size:] == 0xEE) and gm.canaries_intact()


@pytest.mark.parametrize("C", SIZES)
def test_sizes_and_tails(S, O, C):
    rng = np.random.default_rng(C + 17)
    cover = rng.integers(0, 256, C, dtype=np.uint8)
    for header in (True, False):
        cap = S.stego_capacity(C, S.HEADER_BE32 if header else 0)
        for m in sorted({0, 1, 2, 3, 4, 5, 7, cap // 2, cap - 1, cap}):
            if m < 0 or m > cap:
                continue
            msg = rng.integers(0, 256, m, dtype=np.uint8)
            st, stego = O.stream1_embed(cover, msg, header=header)
            assert st == 0
            for moff in (0, 1, 2, 3):
                _check(S, O, stego, m, header, moff)


def test_bad_headers(S):
    rng = np.random.default_rng(3)
    c = rng.integers(0, 256, 4096, dtype=np.uint8)
    for nbits, cap, want in ((8 * 100 + 1, 1000, S.E_BAD_HEADER), (8 * 600, 1000, S.E_BAD_HEADER),
                             (8 * 300, 299, S.E_MSG_TOO_SMALL), (8 * 300, 300, S.OK)):
        x = c.copy()
        h = format(nbits, "032b")
        for k in range(32):
            x[k] = (x[k] & 0xFE) | int(h[k])
        gs = Guarded(x.size, 0, x)
        gm = Guarded(cap, 0, 0xEE)
        res = S.new_result()
        S.stego_extract_ballot(gs.view, gm.view, 0, S.HEADER_BE32, res)
        r = S.read_result(res)
        assert r["status"] == want
        if want != S.OK:
            assert r["msg_bytes"] == 0 and np.all(gm.host() == 0xEE)


def test_refuses_other_layouts(S):
    st = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    out = torch.zeros(64, dtype=torch.uint8, device="cuda")
    for flags, geom in ((S.LAYOUT_PAPER2, (64, 16, 4, 0)), (S.BITS(2), None),
                        (S.PLANE_ONLY, (64, 16, 4, 0))):
        with pytest.raises(S.StegoError) as e:
            S.stego_extract_ballot(st, out, 8, flags, S.new_result(), geom=geom)
        assert e.value.status == S.E_INVAL


def test_full_size_matches_vector_kernel(S, O):
    """The 8192x8192x3 cover at full capacity: the ballot kernel's message
    equals the oracle's (and so the vector kernel's)."""
    w = synth.single_8192()
    cover = w.cover("cuda")
    msg = w.message("cuda")
    stego = torch.empty_like(cover)
    S.stego_embed(cover, stego, msg, S.HEADER_BE32)
    out = torch.empty(w.msg_bytes, dtype=torch.uint8, device="cuda")
    res = S.new_result()
    S.stego_extract_ballot(stego, out, 0, S.HEADER_BE32, res)
    assert S.read_result(res)["msg_bytes"] == w.msg_bytes
    st, want = O.stream1_extract(stego.cpu().numpy(), cap=w.msg_bytes, header=True)
    assert st == 0 and np.array_equal(out.cpu().numpy(), want)
    assert torch.equal(out, msg)
