"""Dependent launches: every kernel may start launching while the kernel
before it in the stream finishes, and waits (griddepcontrol.wait) before
touching memory.  These chains give the next kernel no host
synchronisation and make it read what the previous one just wrote: one-bit,
k-bit, paper-layout and batched embeds and extracts on the same buffers,
short kernels (a 512x512x3 cover) so that launches overlap as much as they
can.  The final bytes must equal the oracle applied in the same order."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import need_gpu

pytestmark = pytest.mark.gpu

W, H, CH = 512, 512, 3
C = W * H * CH


@pytest.fixture(scope="module")
def S():
    return need_gpu()


@pytest.fixture(scope="module")
def O():
    return oracle.load()


def test_stego_of_stego_chain(S, O):
    """Each embed reads the stego the previous embed wrote (out of place,
    alternating buffers), each extract reads the stego just written."""
    rng = np.random.default_rng(41)
    cover = rng.integers(0, 256, C, dtype=np.uint8)
    cap = S.stego_capacity(C, S.HEADER_BE32)
    msgs = [rng.integers(0, 256, int(rng.integers(1, cap + 1)), dtype=np.uint8)
            for _ in range(24)]
    bufs = [torch.from_numpy(cover).cuda(), torch.empty(C, dtype=torch.uint8, device="cuda")]
    d_msgs = [torch.from_numpy(m).cuda() for m in msgs]
    outs = [torch.full((cap,), 0xEE, dtype=torch.uint8, device="cuda") for _ in msgs]
    res = [S.new_result() for _ in msgs]
    eres = [S.new_result() for _ in msgs]
    torch.cuda.synchronize()
    for i, m in enumerate(d_msgs):
        src, dst = bufs[i % 2], bufs[(i + 1) % 2]
        S.stego_embed(src, dst, m, S.HEADER_BE32 | S.FUSE_STATS, eres[i])
        S.stego_extract(dst, outs[i], 0, S.HEADER_BE32, res[i])
    torch.cuda.synchronize()
    want = cover
    for i, m in enumerate(msgs):
        st, nxt = O.stream1_embed(want, m, header=True)
        assert st == oracle.OK
        r = S.read_result(eres[i])
        assert r["status"] == 0 and (r["changed"], r["sse"]) == O.changed_bytes(want, nxt), i
        want = nxt
    assert np.array_equal(bufs[len(msgs) % 2].cpu().numpy(), want)
    for i, m in enumerate(msgs):
        r = S.read_result(res[i])
        assert r["status"] == 0 and r["msg_bytes"] == m.size, (i, r)
        out = outs[i].cpu().numpy()
        assert np.array_equal(out[:m.size], m) and np.all(out[m.size:] == 0xEE), i


def test_in_place_mixed_chain(S, O):
    """One buffer rewritten in place by one-bit, k-bit one-plane, paper-layout
    and batched embeds in turn, each reading the previous call's bytes."""
    rng = np.random.default_rng(43)
    cover = rng.integers(0, 256, C, dtype=np.uint8)
    buf = torch.from_numpy(cover).cuda()
    geom = (W, H, CH, 1)
    ops = []
    for i in range(16):
        kind = ("s1", "k2plane", "paper", "batched")[i % 4]
        if kind == "s1":
            cap = S.stego_capacity(C, S.HEADER_BE32)
        elif kind == "k2plane":
            cap = S.stego_capacity(C, S.BITS(2) | S.HEADER_BE32 | S.PLANE_ONLY, geom=geom)
        elif kind == "paper":
            cap = (W // 4) * H
        else:
            cap = S.stego_capacity(C, S.HEADER_BE32)
        m = rng.integers(0, 256, int(rng.integers(1, cap + 1)), dtype=np.uint8)
        ops.append((kind, m))
    keep = []
    ws = torch.empty(S.stego_batched_workspace_bytes(1), dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    for kind, m in ops:
        dm = torch.from_numpy(m).cuda()
        r = S.new_result()
        keep += [dm, r]
        if kind == "s1":
            S.stego_embed(buf, buf, dm, S.HEADER_BE32 | S.FUSE_STATS, r)
        elif kind == "k2plane":
            S.stego_embed(buf, buf, dm, S.BITS(2) | S.HEADER_BE32 | S.PLANE_ONLY | S.FUSE_STATS,
                          r, geom=geom)
        elif kind == "paper":
            S.stego_embed(buf, buf, dm, S.LAYOUT_PAPER2 | S.FUSE_STATS, r, geom=geom)
        else:
            d = S.descs_to_device(S.pack_descs([dict(cover=buf, stego=buf, msg=dm,
                                                     cover_bytes=C, msg_bytes=m.size,
                                                     flags=S.HEADER_BE32)]))
            rb = S.new_result(n=1)
            keep += [d, rb]
            S.stego_embed_batched(d, 1, rb, S.FUSE_STATS, ws)
    torch.cuda.synchronize()
    want = cover
    for kind, m in ops:
        if kind in ("s1", "batched"):
            st, want = O.stream1_embed(want, m, header=True)
        elif kind == "k2plane":
            st, want = O.streamk_embed(want, m, 2, header=True, geom=geom)
        else:
            st, want = O.paper2_embed(want, W, H, CH, 1, m)
        assert st == oracle.OK
    assert np.array_equal(buf.cpu().numpy(), want)
