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


def test_destroyed_and_recreated_streams(S, O):
    """Streams created, given one fused-statistics embed each and destroyed
    while that embed may still be queued or running, 300 times in a row: the
    driver may hand a new stream the handle of a destroyed one, and each
    embed still gets its own totals (slots are keyed by the never-reused stream
    ID; past the 256th stream the zeroing path takes over)."""
    import ctypes
    cu = ctypes.CDLL("libcuda.so.1")
    cu.cuStreamCreate.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_uint]
    cu.cuStreamDestroy_v2.argtypes = [ctypes.c_void_p]
    cases = [_case(40 + i, (1 << 20) + 16 * i, fill=0.3 + 0.2 * i) for i in range(4)]
    wants = [_want(O, c, m, {}) for c, m in cases]
    dev = [(torch.from_numpy(c).cuda(), torch.from_numpy(m).cuda()) for c, m in cases]
    n = 300
    outs = [torch.empty_like(dev[i % 4][0]) for i in range(n)]
    res = S.new_result(n=n)
    res.fill_(-1)
    delay_src = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    delay_dst = torch.empty_like(delay_src)
    torch.cuda.synchronize()
    for i in range(n):
        h = ctypes.c_void_p()
        assert cu.cuStreamCreate(ctypes.byref(h), 1) == 0  # non-blocking stream
        ext = torch.cuda.ExternalStream(h.value)
        with torch.cuda.stream(ext):
            delay_dst.copy_(delay_src)  # keeps the embed queued past the destroy
        c, m = dev[i % 4]
        S.stego_embed(c, outs[i], m, S.HEADER_BE32 | S.FUSE_STATS, res[i], stream=h.value)
        assert cu.cuStreamDestroy_v2(h) == 0
    torch.cuda.synchronize()
    rr = S.read_result(res)
    for i in range(n):
        want, stats = wants[i % 4]
        assert rr[i]["status"] == 0 and (rr[i]["changed"], rr[i]["sse"]) == stats, i
        assert np.array_equal(outs[i].cpu().numpy(), want), i
