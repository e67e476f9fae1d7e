"""The continuous-batching server: every request's result is the same alone
and in the mix (bit for bit, tolerance 0), admission never exceeds the
budget, and bad requests complete with an error instead of hanging."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import need_gpu
from paper_0912_0947_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    return need_gpu()


class Pool:
    """Covers of uneven sizes resident on the device, their pre-embedded
    stegos, and one distinct output slot per request."""

    def __init__(self, S, rng, n_covers, n_req, embed_frac=0.7):
        items = synth.uneven_batch(n_covers, seed=int(rng.integers(1 << 30)), lo=16, hi=700)
        self.sizes = [it.cover_bytes for it in items]
        self.mlen = [it.msg_bytes for it in items]
        self.covers = [torch.from_numpy(rng.integers(0, 256, c, dtype=np.uint8)).cuda()
                       for c in self.sizes]
        self.msgs = [torch.from_numpy(rng.integers(0, 256, m, dtype=np.uint8)).cuda()
                     for m in self.mlen]
        self.stegos = []
        for c, m in zip(self.covers, self.msgs):
            s = torch.empty_like(c)
            S.stego_embed(c, s, m, S.HEADER_BE32)
            self.stegos.append(s)
        self.ops = (rng.random(n_req) >= embed_frac).astype(int)  # 0 embed, 1 extract
        self.ids = rng.integers(0, n_covers, n_req)
        self.out = []
        recs = []
        for r in range(n_req):
            i = int(self.ids[r])
            if self.ops[r] == 0:
                o = torch.full((self.sizes[i],), 0x5A, dtype=torch.uint8, device="cuda")
                recs.append(dict(op=S.OP_EMBED, flags=S.HEADER_BE32, cover=self.covers[i],
                                 stego=o, msg=self.msgs[i], cover_bytes=self.sizes[i],
                                 msg_bytes=self.mlen[i]))
            else:
                o = torch.full((self.mlen[i] + 3,), 0xEE, dtype=torch.uint8, device="cuda")
                recs.append(dict(op=S.OP_EXTRACT, flags=S.HEADER_BE32, cover=self.stegos[i],
                                 msg=o, cover_bytes=self.sizes[i], msg_bytes=self.mlen[i] + 3))
            self.out.append(o)
        self.reqs = S.Server.requests(recs)
        for r in range(n_req):
            self.reqs[r]["tag"] = r

    def reset_outputs(self):
        for r, o in enumerate(self.out):
            o.fill_(0x5A if self.ops[r] == 0 else 0xEE)

    def snapshot(self):
        torch.cuda.synchronize()
        return [o.clone() for o in self.out]


def _by_tag(comps):
    return {int(c["tag"]): c for c in comps}


def test_alone_equals_mix(S):
    rng = np.random.default_rng(31)
    n_req = 400
    pool = Pool(S, rng, 48, n_req)
    # alone: one request at a time on a one-slot, batch-of-one server
    srv = S.Server(slots=1, max_batch=1, budget_bytes=1 << 34)
    alone = []
    for r in range(n_req):
        srv.submit(pool.reqs[r:r + 1])
        srv.drain(30)
        alone.extend(srv.poll())
    srv.close()
    a_out = pool.snapshot()
    a = _by_tag(alone)
    assert len(a) == n_req and all(c["batch_size"] == 1 for c in alone)
    # mix: open-loop Poisson arrivals, four slots, batches of up to 64
    pool.reset_outputs()
    srv = S.Server(slots=4, max_batch=64, budget_bytes=1 << 34)
    arrivals = synth.poisson_arrivals(200000.0, n_req, 77)
    comps = srv.run_open_loop(pool.reqs, arrivals, timeout_s=60)
    st = srv.stats()
    srv.close()
    m = _by_tag(comps)
    assert sorted(m) == list(range(n_req))
    for r in range(n_req):
        for k in ("status", "changed", "sse", "msg_bytes"):
            assert int(m[r][k]) == int(a[r][k]), (r, k)
        assert int(m[r]["status"]) == 0
    m_out = pool.snapshot()
    for r in range(n_req):
        assert torch.equal(m_out[r], a_out[r]), r
    # the mix really batched and overlapped: some batch was launched (on
    # another slot, as a slot runs one batch at a time) before an earlier
    # batch had been seen to complete
    assert max(int(c["batch_size"]) for c in comps) > 1
    assert st["batches"] < n_req
    spans = {}
    for c in comps:
        t0, t1 = float(c["t_dispatch"]), float(c["t_done"])
        spans[t0] = max(spans.get(t0, t1), t1)
    order = sorted(spans.items())
    in_flight = max(sum(1 for t0, t1 in order if t0 <= d < t1) for d, _ in order)
    assert len(order) == st["batches"]
    assert in_flight >= 2, "no two batches were ever in flight at once"
    # every request against the oracle: embeds byte for byte with changed
    # and sse, extracts against the oracle's extraction of the same stego
    O = oracle.load()
    for r in range(n_req):
        i = int(pool.ids[r])
        c = pool.covers[i].cpu().numpy()
        msg = pool.msgs[i].cpu().numpy()
        got = m_out[r].cpu().numpy()
        if pool.ops[r] == 0:
            stt, want = O.stream1_embed(c, msg, header=True)
            assert stt == 0 and np.array_equal(got, want), r
            assert (int(m[r]["changed"]), int(m[r]["sse"])) == O.changed_bytes(c, want), r
            assert int(m[r]["msg_bytes"]) == msg.size
        else:
            stt, want = O.stream1_extract(pool.stegos[i].cpu().numpy(), cap=msg.size + 3,
                                          header=True)
            assert stt == 0 and int(m[r]["msg_bytes"]) == want.size == msg.size, r
            assert np.array_equal(got[: want.size], want), r
            assert np.all(got[want.size:] == 0xEE), r


def test_budget_and_bad_requests(S):
    rng = np.random.default_rng(32)
    C = 1 << 20
    covers = [torch.from_numpy(rng.integers(0, 256, C, dtype=np.uint8)).cuda() for _ in range(6)]
    msg = torch.from_numpy(rng.integers(0, 256, 1000, dtype=np.uint8)).cuda()
    outs = [torch.empty(C, dtype=torch.uint8, device="cuda") for _ in range(6)]
    recs = [dict(op=S.OP_EMBED, flags=S.HEADER_BE32, cover=covers[i], stego=outs[i], msg=msg,
                 cover_bytes=C, msg_bytes=1000, tag=i) for i in range(6)]
    big = torch.empty(8 * C, dtype=torch.uint8, device="cuda")
    recs.append(dict(op=S.OP_EMBED, flags=S.HEADER_BE32, cover=big, stego=big, msg=msg,
                     cover_bytes=8 * C, msg_bytes=1000, tag=100))          # over the budget
    recs.append(dict(op=99, cover=covers[0], cover_bytes=C, tag=101))       # unknown op
    recs.append(dict(op=S.OP_EMBED, flags=S.HEADER_BE32, cover=covers[1], stego=outs[1], msg=msg,
                     cover_bytes=C, msg_bytes=C // 8, tag=102))            # too long a message
    recs.append(dict(op=S.OP_EMBED, flags=S.LAYOUT_PAPER2, cover=covers[2], stego=outs[2],
                     msg=msg, cover_bytes=C, msg_bytes=10, tag=103))       # no geometry
    spare = [torch.full((C,), 0x5A, dtype=torch.uint8, device="cuda") for _ in range(2)]
    recs.append(dict(op=S.OP_EMBED, flags=S.BITS(2) | S.PLANE_ONLY | S.HEADER_BE32,
                     cover=covers[2], stego=spare[0], msg=msg, cover_bytes=C, msg_bytes=10,
                     tag=104))  # one plane without a geometry: refused by the single-cover call
    recs.append(dict(op=S.OP_EMBED, flags=S.BITS(3) | S.HEADER_BE32, cover=covers[2],
                     stego=spare[1], msg=msg, cover_bytes=2048, msg_bytes=1000,
                     tag=105))  # k = 3: 2048 bytes carry 764 message bytes, refused
    budget = 5 * C  # two embeds of 2C + 1000 fit, a third does not
    srv = S.Server(slots=3, max_batch=8, budget_bytes=budget)
    srv.submit(S.Server.requests(recs))
    srv.drain(30)
    comps = _by_tag(srv.poll())
    st = srv.stats()
    srv.close()
    assert sorted(comps) == list(range(6)) + [100, 101, 102, 103, 104, 105]
    for i in range(6):
        assert int(comps[i]["status"]) == 0
    assert int(comps[100]["status"]) == S.E_NOMEM
    assert int(comps[101]["status"]) == S.E_INVAL
    assert int(comps[102]["status"]) == S.E_CAPACITY
    assert int(comps[103]["status"]) == S.E_INVAL
    assert int(comps[104]["status"]) == S.E_INVAL
    assert int(comps[105]["status"]) == S.E_CAPACITY
    assert all(bool((t == 0x5A).all()) for t in spare)
    assert 0 < st["peak_in_flight_bytes"] <= budget
    assert st["outstanding"] == 0
    torch.cuda.synchronize()
    ref = torch.empty(C, dtype=torch.uint8, device="cuda")
    S.stego_embed(covers[3], ref, msg, S.HEADER_BE32)
    assert torch.equal(ref, outs[3])


def test_server_config_errors(S):
    for cfg in (dict(slots=0), dict(slots=17), dict(max_batch=0), dict(max_batch=9000),
                dict(budget_bytes=0)):
        kw = dict(slots=2, max_batch=8, budget_bytes=1 << 20)
        kw.update(cfg)
        with pytest.raises(S.StegoError):
            S.Server(**kw)


def test_paper_layout_requests(S):
    """Requests in the paper's layout (Sections VI/VII: one plane, two bits
    per byte, out-of-band length) carry their geometry and are served mixed
    with one-bit stream requests; every result equals the oracle's."""
    O = oracle.load()
    rng = np.random.default_rng(33)
    geoms = [(1920, 12, 3, 0), (33, 7, 3, 2), (64, 16, 4, 3), (1024, 3, 1, 0), (9, 4, 3, 1)]
    recs, want, keep = [], [], []
    for i in range(40):
        W, H, ch, pl = geoms[i % len(geoms)]
        n = W * H * ch
        cov = rng.integers(0, 256, n, dtype=np.uint8)
        N = int(rng.integers(1, (W // 4) * H + 1))
        msg = rng.integers(0, 256, N, dtype=np.uint8)
        c = torch.from_numpy(cov).cuda()
        m = torch.from_numpy(msg).cuda()
        st, w = O.paper2_embed(cov, W, H, ch, pl, msg)
        assert st == 0
        geo = dict(width=W, height=H, channels=ch, plane=pl)
        if i % 2 == 0:
            o = torch.full((n,), 0x5A, dtype=torch.uint8, device="cuda")
            recs.append(dict(op=S.OP_EMBED, flags=S.LAYOUT_PAPER2, cover=c, stego=o, msg=m,
                             cover_bytes=n, msg_bytes=N, **geo))
            want.append(("embed", o, w, O.changed_bytes(cov, w), N))
        else:
            stg = torch.from_numpy(w).cuda()
            o = torch.full((N + 3,), 0xEE, dtype=torch.uint8, device="cuda")
            recs.append(dict(op=S.OP_EXTRACT, flags=S.LAYOUT_PAPER2, cover=stg, msg=o,
                             cover_bytes=n, msg_bytes=N + 3, msg_len=N, **geo))
            want.append(("extract", o, msg, None, N))
            keep.append(stg)
        keep += [c, m, o]
        # a one-bit stream request between the paper-layout ones
        cs = torch.from_numpy(rng.integers(0, 256, 4096, dtype=np.uint8)).cuda()
        ms = torch.from_numpy(rng.integers(0, 256, 100, dtype=np.uint8)).cuda()
        os_ = torch.empty_like(cs)
        keep += [cs, ms, os_]
        recs.append(dict(op=S.OP_EMBED, flags=S.HEADER_BE32, cover=cs, stego=os_, msg=ms,
                         cover_bytes=4096, msg_bytes=100))
    srv = S.Server(slots=3, max_batch=16, budget_bytes=1 << 32)
    arrivals = synth.poisson_arrivals(100000.0, len(recs), 5)
    # the open-loop runner tags completion k with request index k: paper
    # request i is request 2i, the stream request after it 2i + 1
    comps = _by_tag(srv.run_open_loop(S.Server.requests(recs), arrivals, timeout_s=60))
    srv.close()
    for i, (kind, o, w, stats, N) in enumerate(want):
        c = comps[2 * i]
        assert int(c["status"]) == 0 and int(c["msg_bytes"]) == N, (i, c)
        got = o.cpu().numpy()
        if kind == "embed":
            assert np.array_equal(got, w), i
            assert (int(c["changed"]), int(c["sse"])) == stats, i
        else:
            assert np.array_equal(got[:N], w) and np.all(got[N:] == 0xEE), i
    assert all(int(comps[2 * i + 1]["status"]) == 0 and int(comps[2 * i + 1]["msg_bytes"]) == 100
               for i in range(40))


def test_kbit_and_plane_requests(S):
    """Stream-layout requests with k = 2..4 bits per byte and with one
    carrying plane (k = 1, 2 on RGB covers), embed and extract, served in
    the same batches as one-bit requests; every output and statistic equals
    the oracle's."""
    O = oracle.load()
    rng = np.random.default_rng(44)
    kinds = [(2, None), (3, None), (4, None), (1, (64, 33, 3, 1)), (2, (100, 7, 3, 0)),
             (3, (16, 16, 4, 3))]
    recs, want, keep = [], [], []
    for i in range(48):
        k, geom = kinds[i % len(kinds)]
        n = geom[0] * geom[1] * geom[2] if geom else int(rng.integers(40, 20000))
        cov = rng.integers(0, 256, n, dtype=np.uint8)
        flags = S.BITS(k) | S.HEADER_BE32 | (S.PLANE_ONLY if geom else 0)
        cap = S.stego_capacity(n, flags, geom=geom)
        m = int(rng.integers(0, cap + 1))
        msg = rng.integers(0, 256, m, dtype=np.uint8)
        st, w = O.streamk_embed(cov, msg, k, header=True, geom=geom)
        assert st == oracle.OK
        geo = dict(width=geom[0], height=geom[1], channels=geom[2], plane=geom[3]) if geom else {}
        c = torch.from_numpy(cov).cuda()
        if i % 2 == 0:
            mt = torch.from_numpy(msg).cuda()
            o = torch.full((n,), 0x5A, dtype=torch.uint8, device="cuda")
            recs.append(dict(op=S.OP_EMBED, flags=flags, cover=c, stego=o, msg=mt,
                             cover_bytes=n, msg_bytes=m, **geo))
            want.append(("embed", o, w, O.changed_bytes(cov, w), m))
            keep += [c, mt, o]
        else:
            stg = torch.from_numpy(w).cuda()
            o = torch.full((m + 3,), 0xEE, dtype=torch.uint8, device="cuda")
            recs.append(dict(op=S.OP_EXTRACT, flags=flags, cover=stg, msg=o,
                             cover_bytes=n, msg_bytes=m + 3, **geo))
            want.append(("extract", o, msg, None, m))
            keep += [stg, o]
        # a one-bit request between them
        cs = torch.from_numpy(rng.integers(0, 256, 4096, dtype=np.uint8)).cuda()
        ms = torch.from_numpy(rng.integers(0, 256, 100, dtype=np.uint8)).cuda()
        os_ = torch.empty_like(cs)
        keep += [cs, ms, os_]
        recs.append(dict(op=S.OP_EMBED, flags=S.HEADER_BE32, cover=cs, stego=os_, msg=ms,
                         cover_bytes=4096, msg_bytes=100))
    srv = S.Server(slots=3, max_batch=16, budget_bytes=1 << 32)
    arrivals = synth.poisson_arrivals(100000.0, len(recs), 6)
    comps = _by_tag(srv.run_open_loop(S.Server.requests(recs), arrivals, timeout_s=60))
    srv.close()
    for i, (kind, o, w, stats, m) in enumerate(want):
        c = comps[2 * i]
        assert int(c["status"]) == 0 and int(c["msg_bytes"]) == m, (i, c)
        got = o.cpu().numpy()
        if kind == "embed":
            assert np.array_equal(got, w), i
            assert (int(c["changed"]), int(c["sse"])) == stats, i
        else:
            assert np.array_equal(got[:m], w) and np.all(got[m:] == 0xEE), i
    assert all(int(comps[2 * i + 1]["status"]) == 0 for i in range(48))
    assert max(int(c["batch_size"]) for c in comps.values()) > 1
