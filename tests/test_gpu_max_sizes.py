"""Maximum sizes: the longest message the 32-bit header can count (2^29 - 1
bytes, a header value of 2^32 - 8 bits) in a cover of more than 2^32 bytes,
through the single-cover calls and in a batch beside small covers, against
the oracle byte for byte; one byte more is refused before anything is
written, whatever the cover's size."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import need_gpu
from paper_0912_0947_gb300 import synth

pytestmark = pytest.mark.gpu

M_MAX = (1 << 29) - 1                 # header value 8 * M_MAX = 2^32 - 8
T_MAX = 8 * (M_MAX + 4)               # 4,294,967,320 carrying bytes > 2^32
C_BIG = T_MAX + 4099                  # a ragged tail past the carrying bytes


@pytest.fixture(scope="module")
def S():
    return need_gpu()


@pytest.fixture(scope="module")
def big(S):
    cover = synth.uniform_bytes(C_BIG, synth.substream(synth.SEED_BASE + 9, 1), "cuda")
    msg = synth.uniform_bytes(M_MAX, synth.substream(synth.SEED_BASE + 9, 2), "cuda")
    O = oracle.load()
    cov_h, msg_h = cover.cpu().numpy(), msg.cpu().numpy()
    st, want = O.stream1_embed(cov_h, msg_h, header=True)
    assert st == oracle.OK
    return cover, msg, cov_h, msg_h, want, O.changed_bytes(cov_h, want)


def test_largest_header_message_single_cover(S, big):
    cover, msg, cov_h, msg_h, want, stats = big
    assert S.stego_capacity(C_BIG, S.HEADER_BE32) == M_MAX
    stego = torch.empty_like(cover)
    res = S.new_result()
    S.stego_embed(cover, stego, msg, S.HEADER_BE32 | S.FUSE_STATS, res)
    r = S.read_result(res)
    assert r["status"] == 0 and r["msg_bytes"] == M_MAX
    assert (r["changed"], r["sse"]) == stats
    assert np.array_equal(stego.cpu().numpy(), want)
    out = torch.full((M_MAX + 16,), 0xEE, dtype=torch.uint8, device="cuda")
    res2 = S.new_result()
    S.stego_extract(stego, out, 0, S.HEADER_BE32, res2)
    r2 = S.read_result(res2)
    assert r2["status"] == 0 and r2["msg_bytes"] == M_MAX
    assert torch.equal(out[:M_MAX], msg) and bool((out[M_MAX:] == 0xEE).all())
    # one byte more does not fit the header's count: refused, nothing written
    mark = torch.full((64,), 0x5A, dtype=torch.uint8, device="cuda")
    big_msg = torch.empty(M_MAX + 1, dtype=torch.uint8, device="cuda")
    with pytest.raises(S.StegoError) as e:
        S.stego_embed(cover, stego, big_msg, S.HEADER_BE32, mark[:32].view(torch.int64))
    assert e.value.status == S.E_CAPACITY
    assert bool((mark == 0x5A).all())


def test_largest_header_message_in_a_batch(S, big):
    cover, msg, cov_h, msg_h, want, stats = big
    rng = np.random.default_rng(9)
    small = [torch.from_numpy(rng.integers(0, 256, n, dtype=np.uint8)).cuda()
             for n in (40, 4096, 70001)]
    small_msg = [torch.from_numpy(rng.integers(0, 256, c.numel() // 8 - 4, dtype=np.uint8)).cuda()
                 for c in small]
    stego = torch.empty_like(cover)
    small_out = [torch.empty_like(c) for c in small]
    covers = [small[0], cover, small[1], small[2]]
    stegos = [small_out[0], stego, small_out[1], small_out[2]]
    msgs = [small_msg[0], msg, small_msg[1], small_msg[2]]
    recs = [dict(cover=c, stego=s_, msg=m, cover_bytes=c.numel(), msg_bytes=m.numel(),
                 flags=S.HEADER_BE32) for c, s_, m in zip(covers, stegos, msgs)]
    n = len(recs)
    descs = S.descs_to_device(S.pack_descs(recs))
    res = S.new_result(n=n)
    ws = torch.empty(S.stego_batched_workspace_bytes(n), dtype=torch.uint8, device="cuda")
    S.stego_embed_batched(descs, n, res, S.FUSE_STATS, ws)
    rr = S.read_result(res)
    assert all(r["status"] == 0 for r in rr)
    assert rr[1]["msg_bytes"] == M_MAX and (rr[1]["changed"], rr[1]["sse"]) == stats
    assert np.array_equal(stego.cpu().numpy(), want)
    O = oracle.load()
    for i in (0, 2, 3):
        st, w = O.stream1_embed(covers[i].cpu().numpy(), msgs[i].cpu().numpy(), header=True)
        assert st == 0 and np.array_equal(stegos[i].cpu().numpy(), w), i
    outs = [torch.empty(m.numel() + 8, dtype=torch.uint8, device="cuda") for m in msgs]
    xr = [dict(cover=s_, msg=o, cover_bytes=s_.numel(), msg_bytes=o.numel(),
               flags=S.HEADER_BE32) for s_, o in zip(stegos, outs)]
    S.stego_extract_batched(S.descs_to_device(S.pack_descs(xr)), n, res, 0, ws)
    rx = S.read_result(res)
    assert all(r["status"] == 0 and r["msg_bytes"] == m.numel() for r, m in zip(rx, msgs))
    assert all(torch.equal(o[:m.numel()], m) for o, m in zip(outs, msgs))
