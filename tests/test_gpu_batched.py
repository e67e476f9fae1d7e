"""GPU parity of the persistent batched path: every descriptor's output and
result equal the oracle's and the single-cover call's, including covers of
uneven sizes, in-place and misaligned buffers, empty covers and per-cover
errors; a captured CUDA graph replays the same work."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import need_gpu, pmap
from paper_0912_0947_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    return need_gpu()


@pytest.fixture(scope="module")
def O():
    return oracle.load()


class Arena:
    """One device buffer holding many covers at chosen offsets."""

    def __init__(self, sizes, offs, fill=None, device="cuda"):
        self.pos = []
        p = 0
        for n, o in zip(sizes, offs):
            p = (p + 255) // 256 * 256 + o
            self.pos.append(p)
            p += n
        self.buf = torch.zeros(p + 256, dtype=torch.uint8, device=device)
        self.sizes = list(sizes)
        if fill is not None:
            for i, a in enumerate(fill):
                self.view(i).copy_(torch.from_numpy(np.ascontiguousarray(a)).to(device))

    def view(self, i):
        return self.buf[self.pos[i]: self.pos[i] + self.sizes[i]]


def _mixed_batch(rng, count):
    items = []
    for i in range(count):
        C = int(rng.choice([0, 7, 31, 32, 40, 4096, 65536, 65536 * 3 + 17,
                            int(rng.integers(1, 300000))]))
        header = bool(rng.integers(0, 2))
        cap = max(C // 8 - (4 if header else 0), 0)
        if header and C < 32:
            m = 0
        else:
            m = int(rng.integers(0, cap + 1)) if cap else 0
        if i % 11 == 5:
            m = cap + 1  # a capacity error for this cover only
        items.append(dict(C=C, header=header, m=m,
                          inplace=bool(i % 3 == 0),
                          coff=int(rng.choice([0, 0, 0, 5])),
                          moff=int(rng.choice([0, 1]))))
    return items


def _run_embed(S, items, rng, stats=True):
    covers = [rng.integers(0, 256, it["C"], dtype=np.uint8) for it in items]
    msgs = [rng.integers(0, 256, it["m"], dtype=np.uint8) for it in items]
    ca = Arena([it["C"] for it in items], [it["coff"] for it in items], covers)
    sa = Arena([it["C"] for it in items], [it["coff"] for it in items])
    ma = Arena([it["m"] for it in items], [it["moff"] for it in items], msgs)
    recs = []
    for i, it in enumerate(items):
        st = ca.view(i) if it["inplace"] else sa.view(i)
        recs.append(dict(cover=ca.view(i), stego=st, msg=ma.view(i), cover_bytes=it["C"],
                         msg_bytes=it["m"], flags=S.HEADER_BE32 if it["header"] else 0))
    descs = S.descs_to_device(S.pack_descs(recs))
    n = len(items)
    res = S.new_result(n=n)
    ws = torch.empty(S.stego_batched_workspace_bytes(n), dtype=torch.uint8, device="cuda")
    S.stego_embed_batched(descs, n, res, S.FUSE_STATS if stats else 0, ws)
    torch.cuda.synchronize()
    outs = [(ca.view(i) if it["inplace"] else sa.view(i)) for i, it in enumerate(items)]
    return covers, msgs, outs, S.read_result(res), (ca, sa, ma, descs, res, ws)


def test_batched_embed_extract_matches_oracle(S, O):
    rng = np.random.default_rng(21)
    items = _mixed_batch(rng, 120)
    covers, msgs, outs, results, keep = _run_embed(S, items, rng)
    stegos = []
    for i, it in enumerate(items):
        st, want = O.stream1_embed(covers[i], msgs[i], header=it["header"])
        r = results[i]
        assert r["status"] == st, (i, it, r)
        if st != oracle.OK:
            assert r["msg_bytes"] == 0
            stegos.append(None)
            continue
        got = outs[i].cpu().numpy()
        assert np.array_equal(got, want), (i, it)
        assert (r["changed"], r["sse"]) == O.changed_bytes(covers[i], want)
        assert r["msg_bytes"] == it["m"]
        stegos.append(want)
    # batched extraction of the same covers into stale buffers
    ok = [i for i in range(len(items)) if stegos[i] is not None]
    sizes = [items[i]["C"] for i in ok]
    sa = Arena(sizes, [items[i]["coff"] for i in ok], [stegos[i] for i in ok])
    caps = [items[i]["m"] + 2 for i in ok]
    ma = Arena(caps, [items[i]["moff"] for i in ok], [np.full(c, 0xEE, np.uint8) for c in caps])
    recs = [dict(cover=sa.view(j), msg=ma.view(j), cover_bytes=sizes[j], msg_bytes=caps[j],
                 msg_len=items[i]["m"], flags=S.HEADER_BE32 if items[i]["header"] else 0)
            for j, i in enumerate(ok)]
    descs = S.descs_to_device(S.pack_descs(recs))
    res = S.new_result(n=len(ok))
    ws = torch.empty(S.stego_batched_workspace_bytes(len(ok)), dtype=torch.uint8, device="cuda")
    S.stego_extract_batched(descs, len(ok), res, 0, ws)
    rr = S.read_result(res)
    for j, i in enumerate(ok):
        assert rr[j]["status"] == 0 and rr[j]["msg_bytes"] == items[i]["m"], (i, rr[j])
        got = ma.view(j).cpu().numpy()
        assert np.array_equal(got[: items[i]["m"]], msgs[i])
        assert np.all(got[items[i]["m"]:] == 0xEE)


def test_batched_equals_single_calls_and_graph_replay(S):
    rng = np.random.default_rng(22)
    items = [dict(C=int(c), header=True, m=int(c) // 8 - 4 - int(k), inplace=False, coff=0, moff=0)
             for c, k in zip(rng.integers(40, 2_000_000, 64), rng.integers(0, 5, 64))]
    covers, msgs, outs, results, keep = _run_embed(S, items, rng)
    for i, it in enumerate(items):
        c = torch.from_numpy(covers[i]).cuda()
        s = torch.empty_like(c)
        r = S.new_result()
        S.stego_embed(c, s, torch.from_numpy(msgs[i]).cuda(), S.HEADER_BE32 | S.FUSE_STATS, r)
        assert torch.equal(s, outs[i]), i
        one = S.read_result(r)
        assert (one["changed"], one["sse"]) == (results[i]["changed"], results[i]["sse"])
    ca, sa, ma, descs, res, ws = keep
    g = S.BatchedGraph(S.OP_EMBED_BATCHED, descs, len(items), res, S.FUSE_STATS, ws)
    sa.buf.zero_()
    res.zero_()
    g.launch()
    g.launch()  # replays are idempotent
    torch.cuda.synchronize()
    again = S.read_result(res)
    for i in range(len(items)):
        assert torch.equal(sa.view(i), outs[i])
        assert again[i] == results[i]
    g.close()


@pytest.mark.parametrize("tile,threads,vec", [(4096, 64, 1), (65536, 256, 4), (1 << 20, 512, 8),
                                              (12288, 128, 2)])
def test_batched_launch_shapes(S, O, tile, threads, vec):
    rng = np.random.default_rng(tile + threads)
    items = _mixed_batch(rng, 40)
    covers = [rng.integers(0, 256, it["C"], dtype=np.uint8) for it in items]
    msgs = [rng.integers(0, 256, it["m"], dtype=np.uint8) for it in items]
    ca = Arena([it["C"] for it in items], [it["coff"] for it in items], covers)
    sa = Arena([it["C"] for it in items], [it["coff"] for it in items])
    ma = Arena([it["m"] for it in items], [it["moff"] for it in items], msgs)
    recs = [dict(cover=ca.view(i), stego=sa.view(i), msg=ma.view(i), cover_bytes=it["C"],
                 msg_bytes=it["m"], flags=S.HEADER_BE32 if it["header"] else 0)
            for i, it in enumerate(items)]
    descs = S.descs_to_device(S.pack_descs(recs))
    res = S.new_result(n=len(items))
    ws = torch.empty(S.stego_batched_workspace_bytes(len(items)), dtype=torch.uint8, device="cuda")
    S.stego_embed_batched(descs, len(items), res, S.FUSE_STATS, ws, tune=(threads, vec, 0, tile))
    rr = S.read_result(res)
    for i, it in enumerate(items):
        st, want = O.stream1_embed(covers[i], msgs[i], header=it["header"])
        assert rr[i]["status"] == st
        if st == 0:
            assert np.array_equal(sa.view(i).cpu().numpy(), want)


def test_batched_argument_errors(S):
    descs = torch.zeros(72, dtype=torch.uint8, device="cuda")
    res = S.new_result(n=1)
    ws = torch.empty(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(S.StegoError) as e:
        S.stego_embed_batched(descs, 1, res, 0, ws)
    assert e.value.status == S.E_NOMEM
    ws = torch.empty(S.stego_batched_workspace_bytes(1), dtype=torch.uint8, device="cuda")
    with pytest.raises(S.StegoError) as e:
        S.stego_extract_batched(descs, 1, res, S.FUSE_STATS, ws)
    assert e.value.status == S.E_INVAL
    # an all-zero descriptor is an empty cover: ok, nothing to do
    S.stego_embed_batched(descs, 1, res, 0, ws)
    assert S.read_result(res)[0]["status"] == 0


def test_video_frames(S, O):
    """600 frames of 1920x1080x3 (gradient plus noise), one message stream
    split across frames at half capacity with a per-frame header, all frames
    in one batched launch: every frame's stego, changed and sse against the
    oracle byte for byte (the oracle on every host core, frame by frame),
    and every frame's batched extraction against the oracle's."""
    v = synth.Video()
    F, fb, P = v.frames, v.frame_bytes, v.per_frame_msg
    frames = v.frame_range(0, F, "cuda").view(F, fb)
    stream = v.message("cuda")
    stego = torch.empty_like(frames)
    recs = [dict(cover=frames[f], stego=stego[f], msg=stream[f * P:(f + 1) * P], cover_bytes=fb,
                 msg_bytes=P, flags=S.HEADER_BE32) for f in range(F)]
    descs = S.descs_to_device(S.pack_descs(recs))
    res = S.new_result(n=F)
    ws = torch.empty(S.stego_batched_workspace_bytes(F), dtype=torch.uint8, device="cuda")
    S.stego_embed_batched(descs, F, res, S.FUSE_STATS, ws)
    rr = S.read_result(res)
    assert all(r["status"] == 0 and r["msg_bytes"] == P for r in rr)
    out = torch.full((F * P,), 0xEE, dtype=torch.uint8, device="cuda")
    recs = [dict(cover=stego[f], msg=out[f * P:(f + 1) * P], cover_bytes=fb, msg_bytes=P,
                 flags=S.HEADER_BE32) for f in range(F)]
    descs_x = S.descs_to_device(S.pack_descs(recs))
    res_x = S.new_result(n=F)
    S.stego_extract_batched(descs_x, F, res_x, 0, ws)
    rx = S.read_result(res_x)
    assert all(r["status"] == 0 and r["msg_bytes"] == P for r in rx)
    fr_h, st_h = frames.cpu().numpy(), stego.cpu().numpy()
    msg_h, out_h = stream.cpu().numpy(), out.cpu().numpy()

    def check(f):
        st, want = O.stream1_embed(fr_h[f], msg_h[f * P:(f + 1) * P], header=True)
        if st != 0 or not np.array_equal(st_h[f], want):
            return "embed"
        if (rr[f]["changed"], rr[f]["sse"]) != O.changed_bytes(fr_h[f], want):
            return "stats"
        xs, xm = O.stream1_extract(st_h[f], cap=P, header=True)
        if xs != 0 or not np.array_equal(out_h[f * P:(f + 1) * P], xm):
            return "extract"
        return None

    bad = [(f, e) for f, e in enumerate(pmap(check, F)) if e]
    assert not bad, bad[:10]
    assert np.array_equal(out_h, msg_h), "concatenated per-frame extracts give the stream back"


def test_uneven_4096_full_size(S, O):
    """4096 covers, sides log-uniform in [64, 4096], 1 or 3 channels,
    messages at 5..100 % of capacity (about 8 GB), in one persistent launch:
    every cover's stego, changed and sse against the oracle byte for byte
    (the oracle on every host core), the padding between covers untouched,
    and every cover's batched extraction against the oracle's."""
    items = synth.uneven_batch(4096)
    sizes = [it.cover_bytes for it in items]
    mlens = [it.msg_bytes for it in items]
    off, moff, p, q = [], [], 0, 0
    for c, m in zip(sizes, mlens):
        off.append(p)
        moff.append(q)
        p += (c + 255) // 256 * 256
        q += (m + 255) // 256 * 256
    covers = synth.uniform_bytes(p, synth.substream(synth.SEED_BASE + 4, 1), "cuda")
    msgs = synth.uniform_bytes(q, synth.substream(synth.SEED_BASE + 4, 2), "cuda")
    stego = covers.clone()  # padding between slots is never written: keep it equal
    n = len(sizes)
    cv = [covers[o:o + c] for o, c in zip(off, sizes)]
    sv = [stego[o:o + c] for o, c in zip(off, sizes)]
    mv = [msgs[o:o + m] for o, m in zip(moff, mlens)]
    descs = S.descs_to_device(S.pack_descs(
        [dict(cover=cv[i], stego=sv[i], msg=mv[i], cover_bytes=sizes[i], msg_bytes=mlens[i],
              flags=S.HEADER_BE32) for i in range(n)]))
    res = S.new_result(n=n)
    ws = torch.empty(S.stego_batched_workspace_bytes(n), dtype=torch.uint8, device="cuda")
    S.stego_embed_batched(descs, n, res, S.FUSE_STATS, ws)
    rr = S.read_result(res)
    assert all(r["status"] == 0 and r["msg_bytes"] == mlens[i] for i, r in enumerate(rr))
    # every differing byte of the arena is a counted change of some cover
    assert int((stego != covers).sum()) == sum(r["changed"] for r in rr)
    out = torch.full_like(msgs, 0xEE)
    ov = [out[o:o + m] for o, m in zip(moff, mlens)]
    descs_x = S.descs_to_device(S.pack_descs(
        [dict(cover=sv[i], msg=ov[i], cover_bytes=sizes[i], msg_bytes=mlens[i],
              flags=S.HEADER_BE32) for i in range(n)]))
    res_x = S.new_result(n=n)
    S.stego_extract_batched(descs_x, n, res_x, 0, ws)
    rx = S.read_result(res_x)
    assert all(r["status"] == 0 and r["msg_bytes"] == mlens[i] for i, r in enumerate(rx))
    cov_h, st_h = covers.cpu().numpy(), stego.cpu().numpy()
    msg_h, out_h = msgs.cpu().numpy(), out.cpu().numpy()

    def check(i):
        o, c, mo, m = off[i], sizes[i], moff[i], mlens[i]
        st, want = O.stream1_embed(cov_h[o:o + c], msg_h[mo:mo + m], header=True)
        if st != 0 or not np.array_equal(st_h[o:o + c], want):
            return "embed"
        if (rr[i]["changed"], rr[i]["sse"]) != O.changed_bytes(cov_h[o:o + c], want):
            return "stats"
        xs, xm = O.stream1_extract(st_h[o:o + c], cap=m, header=True)
        if xs != 0 or not np.array_equal(out_h[mo:mo + m], xm):
            return "extract"
        return None

    bad = [(i, e) for i, e in enumerate(pmap(check, n)) if e]
    assert not bad, bad[:10]


def test_batched_paper_layout_mixed_with_stream(S, O):
    """Paper-layout covers (Sections VI/VII) in the same batches as one-bit
    stream covers: out of place and in place, aligned and misaligned
    buffers, several geometries and planes, per-cover errors; batched
    extraction with the out-of-band length."""
    rng = np.random.default_rng(41)
    geoms = [(16, 5, 3, 1), (1920, 9, 3, 0), (33, 7, 3, 2), (64, 16, 4, 3), (1024, 3, 1, 0),
             (9, 4, 3, 1), (4000, 6, 4, 2), (7, 3, 2, 1), (3, 4, 1, 0), (1920, 20, 3, 1),
             (1920, 30, 3, 2), (512, 40, 3, 2)]
    recs, want, covers, kinds = [], [], [], []
    keep = []
    for gi, (W, H, C, pl) in enumerate(geoms):
        for inplace in (False, True):
            for off in (0, 5):
                n = W * H * C
                cov = rng.integers(0, 256, n, dtype=np.uint8)
                cap = (W // 4) * H
                N = int(rng.integers(0, cap + 1)) if cap else 0
                if gi == 2 and inplace and off == 0:
                    N = cap + 1  # capacity error for this cover only
                msg = rng.integers(0, 256, N, dtype=np.uint8)
                gc = torch.zeros(n + 64, dtype=torch.uint8, device="cuda")
                cv = gc[off:off + n]
                cv.copy_(torch.from_numpy(cov).cuda())
                sv = cv if inplace else torch.full((n + 16,), 0x5A, dtype=torch.uint8,
                                                   device="cuda")[off % 16:off % 16 + n]
                mv = torch.from_numpy(msg).cuda()
                keep += [gc, sv, mv]
                recs.append(dict(cover=cv, stego=sv, msg=mv, cover_bytes=n, msg_bytes=N,
                                 flags=S.LAYOUT_PAPER2, width=W, height=H, channels=C, plane=pl))
                st, w = O.paper2_embed(cov, W, H, C, pl, msg)
                want.append((st, w, cov, msg, sv, (W, H, C, pl)))
    # a few stream-layout covers in the same batch
    for C in (100, 4096, 70001):
        cov = rng.integers(0, 256, C, dtype=np.uint8)
        msg = rng.integers(0, 256, C // 8 - 4, dtype=np.uint8)
        cv = torch.from_numpy(cov).cuda()
        sv = torch.empty_like(cv)
        mv = torch.from_numpy(msg).cuda()
        keep += [cv, sv, mv]
        recs.append(dict(cover=cv, stego=sv, msg=mv, cover_bytes=C, msg_bytes=msg.size,
                         flags=S.HEADER_BE32))
        st, w = O.stream1_embed(cov, msg, header=True)
        want.append((st, w, cov, msg, sv, None))
    n = len(recs)
    for tile in (4096, 65536):
        descs = S.descs_to_device(S.pack_descs(recs))
        res = S.new_result(n=n)
        ws = torch.empty(S.stego_batched_workspace_bytes(n), dtype=torch.uint8, device="cuda")
        # in-place covers are rewritten by the first pass: restore them
        for i, r in enumerate(recs):
            if r["cover"].data_ptr() == r["stego"].data_ptr():
                r["cover"].copy_(torch.from_numpy(want[i][2]).cuda())
        S.stego_embed_batched(descs, n, res, S.FUSE_STATS, ws, tune=(256, 4, 0, tile))
        rr = S.read_result(res)
        for i, (st, w, cov, msg, sv, g) in enumerate(want):
            assert rr[i]["status"] == st, (i, g, rr[i])
            if st != 0:
                continue
            assert np.array_equal(sv.cpu().numpy(), w), (i, g, tile)
            assert (rr[i]["changed"], rr[i]["sse"]) == O.changed_bytes(cov, w), (i, g)
    # batched extraction (paper covers with their out-of-band length)
    xr, xwant = [], []
    for i, (st, w, cov, msg, sv, g) in enumerate(want):
        if st != 0:
            continue
        out = torch.full((msg.size + 3,), 0xEE, dtype=torch.uint8, device="cuda")
        keep.append(out)
        if g is None:
            xr.append(dict(cover=sv, msg=out, cover_bytes=cov.size, msg_bytes=out.numel(),
                           flags=S.HEADER_BE32))
        else:
            W, H, C, pl = g
            xr.append(dict(cover=sv, msg=out, cover_bytes=cov.size, msg_bytes=out.numel(),
                           msg_len=msg.size, flags=S.LAYOUT_PAPER2, width=W, height=H,
                           channels=C, plane=pl))
        xwant.append((msg, out))
    descs = S.descs_to_device(S.pack_descs(xr))
    res = S.new_result(n=len(xr))
    ws = torch.empty(S.stego_batched_workspace_bytes(len(xr)), dtype=torch.uint8, device="cuda")
    S.stego_extract_batched(descs, len(xr), res, 0, ws)
    rr = S.read_result(res)
    for j, (msg, out) in enumerate(xwant):
        assert rr[j]["status"] == 0 and rr[j]["msg_bytes"] == msg.size, (j, rr[j])
        o = out.cpu().numpy()
        assert np.array_equal(o[: msg.size], msg) and np.all(o[msg.size:] == 0xEE), j


def test_batched_paper_layout_video(S, O):
    """600 video frames (1920x1080x3) carrying the message stream in the
    paper's layout (plane 0, 2 bits per byte, 388,796 bytes per frame), one
    batched launch: every frame's stego, changed and sse against the oracle
    byte for byte, and every frame's batched extraction (out-of-band length)
    against the oracle's."""
    v = synth.Video()
    F, fb, P = v.frames, v.frame_bytes, v.per_frame_msg
    frames = v.frame_range(0, F, "cuda").view(F, fb)
    stream = v.message("cuda")
    stego = torch.empty_like(frames)
    geo = dict(width=v.width, height=v.height, channels=3, plane=0)
    recs = [dict(cover=frames[f], stego=stego[f], msg=stream[f * P:(f + 1) * P], cover_bytes=fb,
                 msg_bytes=P, flags=S.LAYOUT_PAPER2, **geo) for f in range(F)]
    descs = S.descs_to_device(S.pack_descs(recs))
    res = S.new_result(n=F)
    ws = torch.empty(S.stego_batched_workspace_bytes(F), dtype=torch.uint8, device="cuda")
    S.stego_embed_batched(descs, F, res, S.FUSE_STATS, ws)
    rr = S.read_result(res)
    assert all(r["status"] == 0 and r["msg_bytes"] == P for r in rr)
    # the single-image one-pass kernel gives the same frame
    one = torch.empty(fb, dtype=torch.uint8, device="cuda")
    S.stego_embed(frames[7], one, stream[7 * P:8 * P], S.LAYOUT_PAPER2,
                  geom=(v.width, v.height, 3, 0))
    assert torch.equal(one, stego[7])
    out = torch.full((F * P,), 0xEE, dtype=torch.uint8, device="cuda")
    recs = [dict(cover=stego[f], msg=out[f * P:(f + 1) * P], cover_bytes=fb, msg_bytes=P,
                 msg_len=P, flags=S.LAYOUT_PAPER2, **geo) for f in range(F)]
    descs = S.descs_to_device(S.pack_descs(recs))
    res_x = S.new_result(n=F)
    S.stego_extract_batched(descs, F, res_x, 0, ws)
    rx = S.read_result(res_x)
    assert all(r["status"] == 0 and r["msg_bytes"] == P for r in rx)
    fr_h, st_h = frames.cpu().numpy(), stego.cpu().numpy()
    msg_h, out_h = stream.cpu().numpy(), out.cpu().numpy()

    def check(f):
        st, want = O.paper2_embed(fr_h[f], v.width, v.height, 3, 0, msg_h[f * P:(f + 1) * P])
        if st != 0 or not np.array_equal(st_h[f], want):
            return "embed"
        if (rr[f]["changed"], rr[f]["sse"]) != O.changed_bytes(fr_h[f], want):
            return "stats"
        xs, xm = O.paper2_extract(st_h[f], v.width, v.height, 3, 0, P)
        if xs != 0 or not np.array_equal(out_h[f * P:(f + 1) * P], xm):
            return "extract"
        return None

    bad = [(f, e) for f, e in enumerate(pmap(check, F)) if e]
    assert not bad, bad[:10]
    assert np.array_equal(out_h, msg_h)


def test_kbit_descriptors_refused_per_cover(S, O):
    """k-bit and one-plane stream descriptors are single-cover only: in a
    batch they get STEGO_E_INVAL in their own result and are not written;
    the other covers of the batch embed normally."""
    rng = np.random.default_rng(77)
    covers = [rng.integers(0, 256, 4096, dtype=np.uint8) for _ in range(3)]
    msgs = [rng.integers(0, 256, 100, dtype=np.uint8) for _ in range(3)]
    flags = [S.HEADER_BE32, S.HEADER_BE32 | S.BITS(2), S.HEADER_BE32 | S.PLANE_ONLY]
    geo = [{}, {}, dict(width=32, height=32, channels=4, plane=0)]
    cv = [torch.from_numpy(c).cuda() for c in covers]
    sv = [torch.full((4096,), 0x5A, dtype=torch.uint8, device="cuda") for _ in range(3)]
    mv = [torch.from_numpy(m).cuda() for m in msgs]
    recs = [dict(cover=cv[i], stego=sv[i], msg=mv[i], cover_bytes=4096, msg_bytes=100,
                 flags=flags[i], **geo[i]) for i in range(3)]
    d = S.descs_to_device(S.pack_descs(recs))
    res = S.new_result(n=3)
    ws = torch.empty(S.stego_batched_workspace_bytes(3), dtype=torch.uint8, device="cuda")
    S.stego_embed_batched(d, 3, res, 0, ws)
    r = S.read_result(res)
    assert r[0]["status"] == S.OK and r[1]["status"] == S.E_INVAL and r[2]["status"] == S.E_INVAL
    st, want = O.stream1_embed(covers[0], msgs[0], header=True)
    assert st == 0 and np.array_equal(sv[0].cpu().numpy(), want)
    assert bool((sv[1] == 0x5A).all()) and bool((sv[2] == 0x5A).all())


def test_uneven_4096_misaligned_full_size(S, O):
    """The 4096-cover uneven batch with every cover 1..15 bytes past a 16-byte
    boundary: a third of the stegos at the cover's misalignment, a third at
    another one, a third in place; messages at odd and even addresses.  The
    misaligned tile space's kernels against the oracle on every cover (stego,
    changed, sse) and every batched extraction from the misaligned stegos."""
    items = synth.uneven_batch(4096)
    rng = np.random.default_rng(4096)
    n = len(items)
    sizes = [it.cover_bytes for it in items]
    mlens = [it.msg_bytes for it in items]
    coff = [int(x) for x in rng.integers(1, 16, n)]
    kind = [i % 3 for i in range(n)]  # 0 same misalignment, 1 another one, 2 in place
    soff = [coff[i] if kind[i] != 1 else int((coff[i] + rng.integers(1, 15)) % 16)
            for i in range(n)]
    moff = [int(x) for x in rng.integers(0, 2, n)]
    cpos, spos, mpos, p, q, r = [], [], [], 0, 0, 0
    for i in range(n):
        cpos.append(p + coff[i])
        spos.append(q + soff[i])
        mpos.append(r + moff[i])
        p += (sizes[i] + 16 + 255) // 256 * 256
        q += (sizes[i] + 16 + 255) // 256 * 256
        r += (mlens[i] + 2 + 255) // 256 * 256
    covers = synth.uniform_bytes(p, synth.substream(synth.SEED_BASE + 4, 1), "cuda")
    orig = covers.clone()
    stego = torch.full((q,), 0x5A, dtype=torch.uint8, device="cuda")
    msgs = synth.uniform_bytes(r, synth.substream(synth.SEED_BASE + 4, 2), "cuda")
    cv = [covers[cpos[i]:cpos[i] + sizes[i]] for i in range(n)]
    sv = [cv[i] if kind[i] == 2 else stego[spos[i]:spos[i] + sizes[i]] for i in range(n)]
    mv = [msgs[mpos[i]:mpos[i] + mlens[i]] for i in range(n)]
    descs = S.descs_to_device(S.pack_descs(
        [dict(cover=cv[i], stego=sv[i], msg=mv[i], cover_bytes=sizes[i], msg_bytes=mlens[i],
              flags=S.HEADER_BE32) for i in range(n)]))
    res = S.new_result(n=n)
    ws = torch.empty(S.stego_batched_workspace_bytes(n), dtype=torch.uint8, device="cuda")
    S.stego_embed_batched(descs, n, res, S.FUSE_STATS, ws)
    rr = S.read_result(res)
    assert all(r_["status"] == 0 and r_["msg_bytes"] == mlens[i] for i, r_ in enumerate(rr))
    out = torch.full((r,), 0xEE, dtype=torch.uint8, device="cuda")
    ov = [out[mpos[i] + 1 - moff[i]:mpos[i] + 1 - moff[i] + mlens[i]] for i in range(n)]
    descs_x = S.descs_to_device(S.pack_descs(
        [dict(cover=sv[i], msg=ov[i], cover_bytes=sizes[i], msg_bytes=mlens[i],
              flags=S.HEADER_BE32) for i in range(n)]))
    res_x = S.new_result(n=n)
    S.stego_extract_batched(descs_x, n, res_x, 0, ws)
    rx = S.read_result(res_x)
    assert all(r_["status"] == 0 and r_["msg_bytes"] == mlens[i] for i, r_ in enumerate(rx))
    orig_h, cov_h, st_h = orig.cpu().numpy(), covers.cpu().numpy(), stego.cpu().numpy()
    msg_h, out_h = msgs.cpu().numpy(), out.cpu().numpy()

    def check(i):
        c = orig_h[cpos[i]:cpos[i] + sizes[i]]
        st, want = O.stream1_embed(c, msg_h[mpos[i]:mpos[i] + mlens[i]], header=True)
        got = cov_h[cpos[i]:cpos[i] + sizes[i]] if kind[i] == 2 else \
            st_h[spos[i]:spos[i] + sizes[i]]
        if st != 0 or not np.array_equal(got, want):
            return "embed"
        if (rr[i]["changed"], rr[i]["sse"]) != O.changed_bytes(c, want):
            return "stats"
        if kind[i] != 2 and not np.array_equal(cov_h[cpos[i]:cpos[i] + sizes[i]], c):
            return "cover written"
        xs, xm = O.stream1_extract(want, cap=mlens[i], header=True)
        o = mpos[i] + 1 - moff[i]
        if xs != 0 or not np.array_equal(out_h[o:o + mlens[i]], xm):
            return "extract"
        return None

    bad = [(i, e) for i, e in enumerate(pmap(check, n)) if e]
    assert not bad, bad[:10]
    # nothing outside the buffers was written
    written = np.zeros(q, bool)
    for i in range(n):
        if kind[i] != 2:
            written[spos[i]:spos[i] + sizes[i]] = True
    assert np.all(st_h[~written] == 0x5A)
