"""One stream-layout cover split among ranks at 16-byte cover offsets
(shard.embed_slice / read_header / extract_slice), each slice in a tensor
of its own as on separate GPUs, run one after another on one GPU: the
slices' stego bytes, summed statistics and extracted message bytes equal
the oracle's embed and extraction of the whole cover."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    return need_gpu()


@pytest.fixture(scope="module")
def O():
    return oracle.load()


def _run_split(S, cover_h, msg_h, world, header, inplace=False):
    from paper_0912_0947_gb300 import shard
    C, m = cover_h.size, msg_h.size
    stego, outs, ch, ss = [], [], 0, 0
    for c0, c1 in shard.cover_slices(C, world):
        lo, hi = shard.slice_message_range(c0, c1, m, header)
        cs = torch.from_numpy(cover_h[c0:c1].copy()).cuda()
        st = cs if inplace else torch.full_like(cs, 0x5A)
        part = torch.from_numpy(msg_h[lo:hi].copy()).cuda() if hi > lo else None
        sl = shard.embed_slice(cs, st, c0, C, m, part, header)
        c, s_ = sl.stats()
        ch, ss = ch + c, ss + s_
        stego.append(st)
    full = torch.cat(stego) if stego else torch.zeros(0, dtype=torch.uint8, device="cuda")
    # extraction, each rank on its own slice (the header from the first 32 bytes)
    mm = shard.read_header(full[:32], C, cap=m) if header else m
    assert mm == m
    for (c0, c1), st in zip(shard.cover_slices(C, world), stego):
        lo, hi = shard.slice_message_range(c0, c1, m, header)
        o = torch.full((hi - lo + 3,), 0xEE, dtype=torch.uint8, device="cuda")
        shard.extract_slice(st, c0, C, m, o, header)
        assert bool((o[hi - lo:] == 0xEE).all())
        outs.append(o[: hi - lo])
    got_msg = torch.cat(outs).cpu().numpy() if outs else np.zeros(0, np.uint8)
    return full.cpu().numpy(), (ch, ss), got_msg


@pytest.mark.parametrize("header", [True, False])
@pytest.mark.parametrize("C", [32 + 16, 4096 + 5, (1 << 20) + 16 * 7 + 3])
def test_split_equals_oracle(S, O, C, header):
    rng = np.random.default_rng(C + header)
    cover = rng.integers(0, 256, C, dtype=np.uint8)
    cap = S.stego_capacity(C, S.HEADER_BE32 if header else 0)
    for m in sorted({0, min(1, cap), cap // 2 + 1, cap}):
        msg = rng.integers(0, 256, m, dtype=np.uint8)
        st, want = O.stream1_embed(cover, msg, header=header)
        assert st == 0
        stats = O.changed_bytes(cover, want)
        for world in (1, 2, 3, 5, 8):
            for inplace in (False, True):
                got, gstats, gmsg = _run_split(S, cover, msg, world, header, inplace)
                assert np.array_equal(got, want), (C, m, world, inplace)
                assert gstats == stats
                assert np.array_equal(gmsg, msg)


def test_split_full_size_equals_one_call(S):
    """The 8192x8192x3 cover at full capacity in 4 slices against the
    single-cover call, on the device."""
    from paper_0912_0947_gb300 import shard, synth
    C = 8192 * 8192 * 3
    cover = synth.uniform_bytes(C, synth.substream(synth.SEED_BASE + 5, 1), "cuda")
    m = S.stego_capacity(C, S.HEADER_BE32)
    msg = synth.uniform_bytes(m, synth.substream(synth.SEED_BASE + 5, 2), "cuda")
    one = torch.empty_like(cover)
    r1 = S.new_result()
    S.stego_embed(cover, one, msg, S.HEADER_BE32 | S.FUSE_STATS, r1)
    want = S.read_result(r1)
    parts, ch, ss = [], 0, 0
    for c0, c1 in shard.cover_slices(C, 4):
        lo, hi = shard.slice_message_range(c0, c1, m)
        st = torch.empty(c1 - c0, dtype=torch.uint8, device="cuda")
        sl = shard.CoverSlice(c0, c1, C, m)
        sl.embed(cover[c0:c1], st, msg[lo:hi])
        c, s_ = sl.stats()
        ch, ss = ch + c, ss + s_
        parts.append(st)
    assert torch.equal(torch.cat(parts), one)
    assert (ch, ss) == (want["changed"], want["sse"])
    assert shard.read_header(parts[0][:32], C) == m
    out = torch.empty(m, dtype=torch.uint8, device="cuda")
    for (c0, c1), st in zip(shard.cover_slices(C, 4), parts):
        lo, hi = shard.slice_message_range(c0, c1, m)
        shard.extract_slice(st, c0, C, m, out[lo:hi])
    assert torch.equal(out, msg)


def test_split_errors(S):
    from paper_0912_0947_gb300 import shard
    C = 1000
    cover = torch.zeros(C, dtype=torch.uint8, device="cuda")
    cap = S.stego_capacity(C, S.HEADER_BE32)
    # a stream past the cover: refused on every slice before any launch
    for c0, c1 in shard.cover_slices(C, 3):
        st = torch.full((c1 - c0,), 0x5A, dtype=torch.uint8, device="cuda")
        with pytest.raises(S.StegoError) as e:
            shard.embed_slice(cover[c0:c1], st, c0, C, cap + 1, None)
        assert e.value.status == S.E_CAPACITY and bool((st == 0x5A).all())
    # a message part of the wrong length, a slice start off the 16-byte grid
    with pytest.raises(ValueError):
        shard.embed_slice(cover[:500], cover[:500], 0, C, cap, None)
    with pytest.raises(ValueError):
        shard.embed_slice(cover[8:500], cover[8:500], 8, C, 0, None)
    # headers: a bit count not a multiple of 8, one past the cover, one past a capacity
    for nbits, cap_arg, status in ((12, None, S.E_BAD_HEADER), (8 * 200, None, S.E_BAD_HEADER),
                                   (8 * 50, 49, S.E_MSG_TOO_SMALL)):
        hdr = torch.tensor(list(nbits.to_bytes(4, "big")), dtype=torch.uint8, device="cuda")
        st = torch.zeros(64, dtype=torch.uint8, device="cuda")
        S.stego_embed(st, st, hdr, 0)
        with pytest.raises(S.StegoError) as e:
            shard.read_header(st, 64 if nbits == 8 * 200 else 1000, cap=cap_arg)
        assert e.value.status == status
