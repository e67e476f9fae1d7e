"""Fused statistics of single-cover embeds: per-stream accumulator slots
(no zeroing copy before the kernel) against the oracle's changed-byte count
and squared error, across repeated calls, concurrent streams, more streams
than slots (the zeroing fallback) and graph capture (the fallback too)."""
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


def _case(seed, C, fill=0.7):
    rng = np.random.default_rng(seed)
    cover = rng.integers(0, 256, C, dtype=np.uint8)
    msg = rng.integers(0, 256, int((C // 8 - 4) * fill), dtype=np.uint8)
    return cover, msg


def _want(O, cover, msg, flags_kw):
    st, out = O.streamk_embed(cover, msg, **flags_kw) if "k" in flags_kw else \
        O.stream1_embed(cover, msg, header=True)
    assert st == 0
    return out, O.changed_bytes(cover, out)


def test_repeated_calls_same_stream(S, O):
    """The slot is cleared by each launch's last CTA: the same call twice,
    then a different cover, each gives its own totals."""
    cases = [_case(1, 1 << 20), _case(1, 1 << 20), _case(2, 3 * 65536 + 48), _case(3, 4096)]
    for cover, msg in cases:
        want, stats = _want(O, cover, msg, {})
        c, m = torch.from_numpy(cover).cuda(), torch.from_numpy(msg).cuda()
        s = torch.empty_like(c)
        res = S.new_result()
        res.fill_(-1)  # stale totals must not leak into the result
        S.stego_embed(c, s, m, S.HEADER_BE32 | S.FUSE_STATS, res)
        r = S.read_result(res)
        assert (r["changed"], r["sse"]) == stats
        assert np.array_equal(s.cpu().numpy(), want)


def test_concurrent_streams(S, O):
    """Eight streams, each embedding its own cover, launched back to back so
    their kernels overlap; every result has its own totals."""
    streams = [torch.cuda.Stream() for _ in range(8)]
    jobs = []
    for i, st in enumerate(streams):
        cover, msg = _case(10 + i, (1 << 21) + 16 * i)
        want, stats = _want(O, cover, msg, {})
        c, m = torch.from_numpy(cover).cuda(), torch.from_numpy(msg).cuda()
        jobs.append((st, c, m, torch.empty_like(c), S.new_result(), want, stats))
    torch.cuda.synchronize()
    for _ in range(3):
        for st, c, m, s, res, _, _ in jobs:
            with torch.cuda.stream(st):
                S.stego_embed(c, s, m, S.HEADER_BE32 | S.FUSE_STATS, res, stream=st)
        torch.cuda.synchronize()
        for st, c, m, s, res, want, stats in jobs:
            r = S.read_result(res)
            assert (r["changed"], r["sse"]) == stats
            assert np.array_equal(s.cpu().numpy(), want)


def test_more_streams_than_slots(S, O):
    """300 streams: those past the slot table fall back to zeroing the
    result first; every call still gives the oracle's totals."""
    cover, msg = _case(40, 65536)
    want, stats = _want(O, cover, msg, {})
    c, m = torch.from_numpy(cover).cuda(), torch.from_numpy(msg).cuda()
    outs = []
    streams = [torch.cuda.Stream() for _ in range(300)]
    for st in streams:
        s = torch.empty_like(c)
        res = S.new_result()
        res.fill_(-1)
        S.stego_embed(c, s, m, S.HEADER_BE32 | S.FUSE_STATS, res, stream=st)
        outs.append((s, res))
    torch.cuda.synchronize()
    for s, res in outs:
        r = S.read_result(res)
        assert (r["changed"], r["sse"]) == stats
    assert np.array_equal(outs[-1][0].cpu().numpy(), want)


def test_other_layouts_use_slots(S, O):
    """k-bit (all bytes and one plane) and the paper layout, twice each on
    one stream."""
    rng = np.random.default_rng(50)
    W, H = 96, 40
    cover = rng.integers(0, 256, W * H * 3, dtype=np.uint8)
    c = torch.from_numpy(cover).cuda()
    for flags, geom, kw in ((S.BITS(2) | S.HEADER_BE32, None, {"k": 2, "header": True}),
                            (S.BITS(3) | S.HEADER_BE32 | S.PLANE_ONLY, (W, H, 3, 1),
                             {"k": 3, "header": True, "geom": (W, H, 3, 1)})):
        cap = S.stego_capacity(cover.size, flags, geom=geom)
        msg = rng.integers(0, 256, cap, dtype=np.uint8)
        st, want = O.streamk_embed(cover, msg, **kw)
        assert st == 0
        stats = O.changed_bytes(cover, want)
        for _ in range(2):
            s = torch.empty_like(c)
            res = S.new_result()
            S.stego_embed(c, s, torch.from_numpy(msg).cuda(), flags | S.FUSE_STATS, res, geom=geom)
            r = S.read_result(res)
            assert (r["changed"], r["sse"]) == stats
            assert np.array_equal(s.cpu().numpy(), want)
    N = (W // 4) * H
    msg = rng.integers(0, 256, N, dtype=np.uint8)
    st, want = O.paper2_embed(cover, W, H, 3, 0, msg)
    assert st == 0
    stats = O.changed_bytes(cover, want)
    for _ in range(2):
        s = torch.empty_like(c)
        res = S.new_result()
        S.stego_embed(c, s, torch.from_numpy(msg).cuda(), S.LAYOUT_PAPER2 | S.FUSE_STATS, res,
                      geom=(W, H, 3, 0))
        r = S.read_result(res)
        assert (r["changed"], r["sse"]) == stats


def test_graph_capture_uses_zeroing(S, O):
    """A captured embed with statistics (zeroing inside the graph) replays
    with the right totals, also next to direct calls on the capture stream."""
    cover, msg = _case(60, 1 << 20)
    want, stats = _want(O, cover, msg, {})
    c, m = torch.from_numpy(cover).cuda(), torch.from_numpy(msg).cuda()
    s = torch.empty_like(c)
    res = S.new_result()
    side = torch.cuda.Stream()
    S.stego_embed(c, s, m, S.HEADER_BE32 | S.FUSE_STATS, res, stream=side)  # warm up
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        S.stego_embed(c, s, m, S.HEADER_BE32 | S.FUSE_STATS, res, stream=side)
    res.fill_(-1)
    s.zero_()
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    r = S.read_result(res)
    assert (r["changed"], r["sse"]) == stats
    assert np.array_equal(s.cpu().numpy(), want)
    s2 = torch.empty_like(c)
    res2 = S.new_result()
    S.stego_embed(c, s2, m, S.HEADER_BE32 | S.FUSE_STATS, res2, stream=side)
    g.replay()
    torch.cuda.synchronize()
    assert (S.read_result(res2)["changed"], S.read_result(res2)["sse"]) == stats
    assert (S.read_result(res)["changed"], S.read_result(res)["sse"]) == stats
