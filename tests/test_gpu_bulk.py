"""GPU parity of the shared-memory staged one-bit stream kernels (bulk
asynchronous copies into a ring of stages) against the CPU oracle, byte for
byte, through the C ABI.  The staged kernels are selected with
stego_set_tune (tile_bytes = ring bytes per CTA); the register kernels are
restored afterwards.

Shapes give 2 to 8 stages and tiles of 1 KiB to 64 KiB; sizes give CTAs
with no tile, one partial tile, and many tiles with a ragged last tile and a
tail that is not a whole vector."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import Guarded, need_gpu
from paper_0912_0947_gb300 import synth
from test_gpu_stream1 import _embed_check, _extract_check, _msgs

pytestmark = pytest.mark.gpu

# (threads, vectors per thread, CTAs per SM, ring bytes): stages = ring / tile
SHAPES = [(256, 4, 0, 65536),    # 16 KiB tiles, 4 stages
          (64, 1, 0, 4096),      # 1 KiB tiles, 4 stages
          (512, 8, 0, 131072),   # 64 KiB tiles, 2 stages
          (128, 2, 2, 32768),    # 4 KiB tiles, 8 stages, 2 CTAs per SM
          (256, 8, 0, 196608)]   # 32 KiB tiles, 6 stages
SIZES = [0, 1, 15, 16, 17, 40, 100, 4096, 4097, 65543, 3 * 16384 * 9 + 8,
         (1 << 20) + 13, 786432]


@pytest.fixture(scope="module")
def S():
    return need_gpu()


@pytest.fixture(scope="module")
def O():
    return oracle.load()


class staged:
    """Installs a staged shape for the single-cover embed and extract."""

    def __init__(self, S, shape):
        self.S, self.shape = S, shape

    def __enter__(self):
        S = self.S
        self.old = (S.stego_get_tune(S.OP_EMBED), S.stego_get_tune(S.OP_EXTRACT))
        S.stego_set_tune(S.OP_EMBED, self.shape)
        S.stego_set_tune(S.OP_EXTRACT, self.shape)
        return self

    def __exit__(self, *exc):
        S = self.S
        S.stego_set_tune(S.OP_EMBED, self.old[0])
        S.stego_set_tune(S.OP_EXTRACT, self.old[1])
        return False


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("header", [True, False])
def test_staged_sizes(S, O, shape, header):
    with staged(S, shape):
        for C in SIZES:
            rng = np.random.default_rng(C * 4 + header * 2 + shape[0])
            cover = rng.integers(0, 256, C, dtype=np.uint8)
            cap = S.stego_capacity(C, S.HEADER_BE32 if header else 0)
            for msg in _msgs(cap, rng):
                for inplace in (False, True):
                    stego = _embed_check(S, O, cover, msg, header, inplace=inplace)
                if stego is not None:
                    _extract_check(S, O, stego, msg.size, header)


@pytest.mark.parametrize("offs", [(0, 0, 1), (0, 0, 3), (16, 32, 1), (1, 1, 0), (0, 5, 2)])
def test_staged_message_alignment_and_fallback(S, O, offs):
    """Odd message addresses (byte loads and stores of the message) and, for
    misaligned covers, the byte kernels behind the same shape."""
    with staged(S, SHAPES[0]):
        for C in (4097, 70001, 3 * 65536 + 40):
            rng = np.random.default_rng(C + sum(offs))
            cover = rng.integers(0, 256, C, dtype=np.uint8)
            for header in (True, False):
                cap = S.stego_capacity(C, S.HEADER_BE32 if header else 0)
                for msg in _msgs(cap, rng):
                    stego = _embed_check(S, O, cover, msg, header, offs=offs)
                    if stego is not None:
                        _extract_check(S, O, stego, msg.size, header, offs=(offs[1], offs[2]))


def test_staged_bad_headers(S):
    rng = np.random.default_rng(21)
    c = rng.integers(0, 256, 4096, dtype=np.uint8)
    with staged(S, SHAPES[1]):
        for nbits, cap, want in ((40 * 8 + 3, 1000, S.E_BAD_HEADER),
                                 (8 * 600, 1000, S.E_BAD_HEADER),   # 32 + 4800 > 4096
                                 (8 * 300, 299, S.E_MSG_TOO_SMALL),
                                 (8 * 300, 300, S.OK)):
            x = c.copy()
            h = format(nbits, "032b")
            for k in range(32):
                x[k] = (x[k] & 0xFE) | int(h[k])
            gs = Guarded(x.size, 0, x)
            gm = Guarded(cap, 0, 0xEE)
            res = S.new_result()
            S.stego_extract(gs.view, gm.view, 0, S.HEADER_BE32, res)
            r = S.read_result(res)
            assert r["status"] == want, (nbits, cap, r)
            got = gm.host()
            if want != S.OK:
                assert r["msg_bytes"] == 0 and np.all(got == 0xEE)
            else:
                bits = (x[32:32 + nbits] & 1).reshape(-1, 8)
                exp = np.packbits(bits, axis=1).ravel()
                assert np.array_equal(got[:nbits // 8], exp)
            assert gm.canaries_intact()


def test_set_tune_zero_tile_restores_register_kernels(S):
    old = S.stego_get_tune(S.OP_EMBED)
    try:
        S.stego_set_tune(S.OP_EMBED, (256, 4, 0, 65536))
        assert S.stego_get_tune(S.OP_EMBED).tile_bytes == 65536
        S.stego_set_tune(S.OP_EMBED, (256, 4, 0, 0))
        assert S.stego_get_tune(S.OP_EMBED).tile_bytes == 0
    finally:
        S.stego_set_tune(S.OP_EMBED, old)


@pytest.mark.parametrize("shape", [(256, 4, 0, 65536), (128, 8, 0, 65536), (512, 4, 0, 98304)])
def test_staged_8192_full_capacity(S, O, shape):
    """The 8192x8192x3 cover at full one-bit capacity through the staged
    kernels, every byte against the oracle, plus in place."""
    w = synth.single_8192()
    cover = w.cover("cuda")
    msg = w.message("cuda")
    stego = torch.empty_like(cover)
    out = torch.empty(w.msg_bytes, dtype=torch.uint8, device="cuda")
    res, res2 = S.new_result(), S.new_result()
    with staged(S, shape):
        S.stego_embed(cover, stego, msg, S.HEADER_BE32 | S.FUSE_STATS, res)
        S.stego_extract(stego, out, 0, S.HEADER_BE32, res2)
        buf = cover.clone()
        S.stego_embed(buf, buf, msg, S.HEADER_BE32)
    c_h, m_h = cover.cpu().numpy(), msg.cpu().numpy()
    st, want = O.stream1_embed(c_h, m_h, header=True)
    assert st == 0
    assert np.array_equal(stego.cpu().numpy(), want)
    r = S.read_result(res)
    assert r["status"] == 0 and (r["changed"], r["sse"]) == O.changed_bytes(c_h, want)
    r2 = S.read_result(res2)
    assert r2["status"] == 0 and r2["msg_bytes"] == w.msg_bytes
    assert np.array_equal(out.cpu().numpy(), m_h)
    assert torch.equal(buf, stego)


class withheld_arrival:
    """Makes every staged CTA's first barrier wait run out after limit_ns
    (each barrier expects one arrival the pipeline never gives), and
    restores normal operation on exit."""

    def __init__(self, S, limit_ns):
        self.S, self.limit_ns = S, limit_ns

    def __enter__(self):
        self.S.stego_test_bounded_wait(self.limit_ns, 1)
        return self

    def __exit__(self, *exc):
        self.S.stego_test_bounded_wait(0, 0)


@pytest.mark.parametrize("shape", [(256, 4, 0, 65536), (128, 2, 2, 32768)])
def test_bounded_wait_runs_out(S, O, shape):
    """Failure detection without a fault: every bounded wait of the staged
    kernels runs out (2 ms), the call reports STEGO_E_TIMEOUT in its result,
    writes no output byte, drains its own copies, and the next normal call on
    the same stream returns the oracle's bytes."""
    C = 4 << 20
    rng = np.random.default_rng(99)
    cover = rng.integers(0, 256, C, dtype=np.uint8)
    msg = rng.integers(0, 256, C // 8 - 4 - 1001, dtype=np.uint8)  # odd length
    st, want = O.stream1_embed(cover, msg, header=True)
    assert st == 0
    c = torch.from_numpy(cover).cuda()
    m = torch.from_numpy(msg).cuda()
    good = torch.from_numpy(want).cuda()
    stream = torch.cuda.Stream()
    with staged(S, shape):
        with withheld_arrival(S, 2_000_000):
            out = torch.full_like(c, 0x5A)
            res = S.new_result()
            S.stego_embed(c, out, m, S.HEADER_BE32 | S.FUSE_STATS, res, stream=stream)
            got = torch.full((msg.size + 8,), 0xEE, dtype=torch.uint8, device="cuda")
            res_x = S.new_result()
            S.stego_extract(good, got, 0, S.HEADER_BE32, res_x, stream=stream)
            stream.synchronize()
            assert S.read_result(res)["status"] == S.E_TIMEOUT
            assert S.read_result(res_x)["status"] == S.E_TIMEOUT
            assert bool((out == 0x5A).all()), "a timed-out embed wrote its stego"
            assert bool((got == 0xEE).all()), "a timed-out extract wrote its message"
        # normal operation again, same stream
        out = torch.full_like(c, 0x5A)
        res = S.new_result()
        S.stego_embed(c, out, m, S.HEADER_BE32 | S.FUSE_STATS, res, stream=stream)
        got = torch.full((msg.size + 8,), 0xEE, dtype=torch.uint8, device="cuda")
        res_x = S.new_result()
        S.stego_extract(out, got, 0, S.HEADER_BE32, res_x, stream=stream)
        stream.synchronize()
        r = S.read_result(res)
        assert r["status"] == 0 and (r["changed"], r["sse"]) == O.changed_bytes(cover, want)
        assert np.array_equal(out.cpu().numpy(), want)
        rx = S.read_result(res_x)
        assert rx["status"] == 0 and rx["msg_bytes"] == msg.size
        g = got.cpu().numpy()
        assert np.array_equal(g[: msg.size], msg) and np.all(g[msg.size:] == 0xEE)


def test_bounded_wait_argument_check(S):
    with pytest.raises(S.StegoError) as e:
        S.stego_test_bounded_wait(0, 2)
    assert e.value.status == S.E_INVAL
    S.stego_test_bounded_wait(0, 0)
