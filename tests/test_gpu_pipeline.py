"""Host-resident covers through the overlapped copy pipeline
(stego_pipeline_*): every job's stego, statistics, read-back and extracted
message against the oracle, byte for byte, for uneven batches cut into many
chunks over two and three slots, both layouts, host stegos in place and out
of place, per-job errors (capacity, a job larger than a slot, a bad header)
that leave the job's output unwritten, and the full-size 8192x8192x3 cover."""
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


def pinned(a):
    t = torch.from_numpy(np.ascontiguousarray(a)) if isinstance(a, np.ndarray) else a
    return t.pin_memory()


def _jobs(S, rng, count, slot_bytes):
    """Jobs of uneven sizes: stream layout (header or raw) and paper layout,
    host stego in place or not, some with a read-back, one over capacity,
    one larger than a slot."""
    jobs = []
    for i in range(count):
        paper = i % 5 == 3
        if paper:
            ch = int(rng.choice([1, 3, 4]))
            W = int(rng.choice([16 * int(rng.integers(1, 60)), int(rng.integers(4, 500))]))
            H = int(rng.integers(1, 40))
            C = W * H * ch
            pl = int(rng.integers(0, ch))
            cap = (W // 4) * H
            flags = S.LAYOUT_PAPER2
            geo = dict(width=W, height=H, channels=ch, plane=pl)
        else:
            C = int(rng.choice([40, 4096, int(rng.integers(32, 600_000)),
                                int(rng.integers(1 << 20, 3 << 20))]))
            header = bool(rng.integers(0, 4))
            cap = C // 8 - (4 if header else 0)
            flags = S.HEADER_BE32 if header else 0
            geo = {}
        m = int(rng.integers(0, cap + 1))
        if i == 7:
            m = cap + 1  # this job alone fails its capacity check
        if i == 11:
            # this job alone is larger than a slot (its read-back makes it a
            # staged job in either mode)
            C = slot_bytes + 4096
            flags, geo, m = S.HEADER_BE32, {}, 100
        jobs.append(dict(C=C, m=m, flags=flags, geo=geo, inplace=bool(i % 3 == 1),
                         readback=bool(i % 4 == 0 or i == 11),
                         cover=rng.integers(0, 256, C, dtype=np.uint8),
                         msg=rng.integers(0, 256, m, dtype=np.uint8)))
    return jobs


def _oracle_embed(O, S, j):
    if j["flags"] == S.LAYOUT_PAPER2:
        g = j["geo"]
        return O.paper2_embed(j["cover"], g["width"], g["height"], g["channels"], g["plane"],
                              j["msg"])
    return O.stream1_embed(j["cover"], j["msg"], header=bool(j["flags"] & S.HEADER_BE32))


def _arena_views(sizes, rng, fill):
    """Views into one pinned host buffer at ascending offsets: holes of 0 to
    300 bytes between them, every third view 16-byte aligned."""
    offs, p = [], 0
    for i, n in enumerate(sizes):
        p += int(rng.integers(0, 300))
        if i % 3 == 0:
            p = (p + 15) // 16 * 16
        offs.append(p)
        p += n
    buf = pinned(torch.full((p + 64,), 0x77, dtype=torch.uint8))
    views = [buf[o:o + n] for o, n in zip(offs, sizes)]
    for v, a in zip(views, fill):
        if a is not None:
            v.copy_(torch.from_numpy(np.ascontiguousarray(a)))
    return buf, views


@pytest.mark.parametrize("slots,max_descs,slot_mb,arena,staged",
                         [(2, 16, 8, False, True), (3, 64, 16, True, True), (1, 8, 4, False, True),
                          (2, 32, 6, True, True), (2, 16, 8, False, False),
                          (3, 32, 6, True, False)])
def test_pipeline_embed_extract_matches_oracle(S, O, slots, max_descs, slot_mb, arena, staged):
    """arena: covers, stegos and messages are views into three pinned
    buffers (neighbouring jobs are copied in as one range, holes included).
    staged: every job through the slots and the copy engines; otherwise the
    jobs without a read-back are zero copy."""
    rng = np.random.default_rng(100 + slots + 10 * arena + 100 * staged)
    slot_bytes = slot_mb << 20
    jobs = _jobs(S, rng, 90, slot_bytes)
    pipe = S.Pipeline(slots=slots, max_descs=max_descs, slot_bytes=slot_bytes,
                      mode=S.PIPE_STAGED if staged else S.PIPE_AUTO)
    if arena:
        cbuf, covers = _arena_views([j["C"] for j in jobs], rng, [j["cover"] for j in jobs])
        mbuf, msgs = _arena_views([j["m"] for j in jobs], rng, [j["msg"] for j in jobs])
        sbuf, sviews = _arena_views([j["C"] for j in jobs], rng,
                                    [np.full(j["C"], 0x5A, np.uint8) for j in jobs])
        stegos = [c if j["inplace"] else v for c, v, j in zip(covers, sviews, jobs)]
    else:
        covers = [pinned(j["cover"].copy()) for j in jobs]
        msgs = [pinned(j["msg"]) for j in jobs]
        stegos = [c if j["inplace"] else pinned(np.full(j["C"], 0x5A, np.uint8))
                  for c, j in zip(covers, jobs)]
    rbs = [pinned(np.full(j["m"] + 3, 0xEE, np.uint8)) if j["readback"] else None
           for j in jobs]
    recs = [dict(cover=covers[i], stego=stegos[i], msg=msgs[i], readback=rbs[i],
                 cover_bytes=j["C"], msg_bytes=j["m"], flags=j["flags"], **j["geo"])
            for i, j in enumerate(jobs)]
    res, rb_res = pipe.embed(S.Pipeline.jobs(recs), S.FUSE_STATS, readback_results=True)

    def check(i):
        j = jobs[i]
        st, want = _oracle_embed(O, S, j)
        r = res[i]
        if i == 11:
            st = S.E_NOMEM
        if r["status"] != st:
            return ("status", r["status"], st)
        got = stegos[i].numpy()
        if st != 0:
            # refused: the host stego (or the in-place cover) is not written
            unchanged = j["cover"] if j["inplace"] else np.full(j["C"], 0x5A, np.uint8)
            return None if np.array_equal(got, unchanged) else "written"
        if not np.array_equal(got, want):
            return "stego"
        if (r["changed"], r["sse"]) != O.changed_bytes(j["cover"], want) or r["msg_bytes"] != j["m"]:
            return "stats"
        if j["readback"]:
            rr = rb_res[i]
            rb = rbs[i].numpy()
            if rr["status"] != 0 or rr["msg_bytes"] != j["m"]:
                return ("readback status", rr)
            if not np.array_equal(rb[: j["m"]], j["msg"]) or not np.all(rb[j["m"]:] == 0xEE):
                return "readback"
        elif rb_res[i]["status"] != 0 or rb_res[i]["msg_bytes"] != 0:
            return "readback result of a job without one"
        return None

    bad = [(i, e) for i, e in enumerate(pmap(check, len(jobs))) if e]
    assert not bad, bad[:10]
    if arena:  # the holes between the views were copied in, never written back
        for buf, views in ((cbuf, covers), (sbuf, sviews), (mbuf, msgs)):
            mask = np.ones(buf.numel(), bool)
            base = buf.data_ptr()
            for v in views:
                mask[v.data_ptr() - base: v.data_ptr() - base + v.numel()] = False
            assert np.all(buf.numpy()[mask] == 0x77)

    # extraction of the stegos, through the pipeline, into stale host buffers
    ok = [i for i in range(len(jobs)) if res[i]["status"] == 0]
    outs = {i: pinned(np.full(jobs[i]["m"] + 5, 0xCD, np.uint8)) for i in ok}
    xrecs = [dict(cover=stegos[i], msg=outs[i], cover_bytes=jobs[i]["C"],
                  msg_bytes=jobs[i]["m"] + 5, msg_len=jobs[i]["m"], flags=jobs[i]["flags"],
                  **jobs[i]["geo"]) for i in ok]
    # a stego whose header claims more bits than it holds: a device-side error
    bad_stego = pinned(np.zeros(4096, np.uint8))
    bad_stego[0] = 1  # header MSB set: 2^31 bits
    bad_out = pinned(np.full(64, 0xCD, np.uint8))
    xrecs.append(dict(cover=bad_stego, msg=bad_out, cover_bytes=4096, msg_bytes=64,
                      flags=S.HEADER_BE32))
    xres = pipe.extract(S.Pipeline.jobs(xrecs))
    pipe.close()
    assert xres[-1]["status"] == S.E_BAD_HEADER and bool((bad_out == 0xCD).all())

    def xcheck(k):
        i = ok[k]
        j = jobs[i]
        st_h = stegos[i].numpy()
        if j["flags"] == S.LAYOUT_PAPER2:
            g = j["geo"]
            st, want = O.paper2_extract(st_h, g["width"], g["height"], g["channels"], g["plane"],
                                        j["m"])
        else:
            st, want = O.stream1_extract(st_h, cap=j["m"] + 5,
                                         header=bool(j["flags"] & S.HEADER_BE32),
                                         raw_len=j["m"])
        r = xres[k]
        if st != 0 or r["status"] != 0 or r["msg_bytes"] != want.size:
            return ("status", r, st)
        got = outs[i].numpy()
        if not np.array_equal(got[: want.size], want) or not np.all(got[want.size:] == 0xCD):
            return "message"
        return None

    bad = [(ok[k], e) for k, e in enumerate(pmap(xcheck, len(ok))) if e]
    assert not bad, bad[:10]


def test_pipeline_full_size_cover(S, O):
    """The 8192x8192x3 cover at full capacity, three jobs through two 256 MiB
    slots with read-backs: every stego and read-back against the oracle."""
    w = synth.single_8192()
    cover = w.cover("cpu").numpy()
    msg = w.message("cpu").numpy()
    st, want = O.stream1_embed(cover, msg, header=True)
    assert st == 0
    pipe = S.Pipeline(slots=2, max_descs=4, slot_bytes=256 << 20)
    c_h, m_h = pinned(cover), pinned(msg)
    outs = [pinned(torch.empty(cover.size, dtype=torch.uint8)) for _ in range(3)]
    rbs = [pinned(torch.empty(msg.size, dtype=torch.uint8)) for _ in range(3)]
    recs = [dict(cover=c_h, stego=outs[k], msg=m_h, readback=rbs[k], cover_bytes=cover.size,
                 msg_bytes=msg.size, flags=S.HEADER_BE32) for k in range(3)]
    res, rb = pipe.embed(S.Pipeline.jobs(recs), S.FUSE_STATS, readback_results=True)
    pipe.close()
    stats = O.changed_bytes(cover, want)
    for k in range(3):
        assert res[k]["status"] == 0 and (res[k]["changed"], res[k]["sse"]) == stats
        assert np.array_equal(outs[k].numpy(), want), k
        assert rb[k]["status"] == 0 and rb[k]["msg_bytes"] == msg.size
        assert np.array_equal(rbs[k].numpy(), msg), k


def test_pipeline_config_and_argument_errors(S):
    for cfg in (dict(slots=0), dict(slots=9), dict(max_descs=0), dict(max_descs=9000),
                dict(slot_bytes=100), dict(mode=2)):
        kw = dict(slots=2, max_descs=8, slot_bytes=1 << 20)
        kw.update(cfg)
        with pytest.raises(S.StegoError):
            S.Pipeline(**kw)
    pipe = S.Pipeline(slots=2, max_descs=8, slot_bytes=1 << 20)
    with pytest.raises(S.StegoError) as e:
        pipe.embed(S.Pipeline.jobs([]), flags=0x4000)
    assert e.value.status == S.E_INVAL
    assert pipe.embed(S.Pipeline.jobs([])) == []
    pipe.close()


def test_pipeline_edge_cases(S, O):
    """Empty covers and messages, a batch whose every job is refused, and a
    job that exactly fills a slot (cover + message + 1280 bytes, staged by
    its read-back) next to one a byte too large."""
    rng = np.random.default_rng(7)
    C, m = 1 << 20, 1000
    slot = C + m + 1280 + (m + 255) // 256 * 256
    pipe = S.Pipeline(slots=2, max_descs=4, slot_bytes=slot, mode=S.PIPE_STAGED)
    cover = rng.integers(0, 256, C + 1, dtype=np.uint8)
    msg = rng.integers(0, 256, m, dtype=np.uint8)
    c_fit, c_big = pinned(cover[:C].copy()), pinned(cover.copy())
    m_h = pinned(msg)
    o_fit = pinned(np.full(C, 0x5A, np.uint8))
    o_big = pinned(np.full(C + 1, 0x5A, np.uint8))
    rb_fit = pinned(np.full(m, 0xEE, np.uint8))
    rb_big = pinned(np.full(m, 0xEE, np.uint8))
    empty = pinned(np.zeros(0, np.uint8))
    recs = [dict(cover=c_fit, stego=o_fit, msg=m_h, readback=rb_fit, cover_bytes=C,
                 msg_bytes=m, flags=S.HEADER_BE32),
            dict(cover=c_big, stego=o_big, msg=m_h, readback=rb_big, cover_bytes=C + 1,
                 msg_bytes=m, flags=S.HEADER_BE32),
            dict(cover=empty, stego=empty, msg=empty, cover_bytes=0, msg_bytes=0, flags=0),
            dict(cover=c_fit, stego=o_fit, msg=empty, cover_bytes=C, msg_bytes=0, flags=0)]
    res, rb = pipe.embed(S.Pipeline.jobs(recs), S.FUSE_STATS, readback_results=True)
    st, want = O.stream1_embed(cover[:C], msg, header=True)
    assert res[0]["status"] == 0 and rb[0]["status"] == 0 and rb[0]["msg_bytes"] == m
    assert res[1]["status"] == S.E_NOMEM and rb[1]["status"] == S.E_NOMEM
    assert bool((o_big == 0x5A).all()) and bool((rb_big == 0xEE).all())
    assert res[2]["status"] == 0 and res[2]["msg_bytes"] == 0
    # the raw empty message leaves the stego equal to the cover
    assert res[3]["status"] == 0 and np.array_equal(o_fit.numpy(), cover[:C])
    assert np.array_equal(rb_fit.numpy(), msg)
    # every job refused: nothing staged, nothing written
    bad = [dict(cover=c_fit, stego=o_big[:C], msg=m_h, cover_bytes=C, msg_bytes=C, flags=0),
           dict(cover=c_fit, stego=o_big[:C], msg=m_h, cover_bytes=C, msg_bytes=m, flags=0x4000)]
    o_big.fill_(0x5A)
    res = pipe.embed(S.Pipeline.jobs(bad))
    assert [r["status"] for r in res] == [S.E_CAPACITY, S.E_INVAL]
    assert bool((o_big == 0x5A).all())
    # an extraction of an empty-message stego (header 0) writes no byte
    st0, w0 = O.stream1_embed(cover[:C], np.zeros(0, np.uint8), header=True)
    s0 = pinned(w0)
    out0 = pinned(np.full(8, 0xCD, np.uint8))
    rx = pipe.extract(S.Pipeline.jobs([dict(cover=s0, msg=out0, cover_bytes=C, msg_bytes=8,
                                            flags=S.HEADER_BE32)]))
    pipe.close()
    assert rx[0]["status"] == 0 and rx[0]["msg_bytes"] == 0 and bool((out0 == 0xCD).all())
