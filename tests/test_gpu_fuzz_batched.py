"""Seeded random batches against the CPU oracle, cover by cover: stream
(header or raw) and paper-layout covers of random sizes and geometries, in
place or not, at random offsets from a 16-byte boundary, some with
messages over capacity (their own status, nothing written), one batched
embed with statistics and one batched extract per batch, at two tile
sizes."""
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


def _batch(S, O, rng, n):
    recs, exts, checks, keep = [], [], [], []
    for _ in range(n):
        paper = rng.random() < 0.35
        ch = int(rng.choice([1, 3, 4])) if paper else 1
        if paper:
            W = int(rng.choice([16 * int(rng.integers(1, 40)), int(rng.integers(1, 300))]))
            H = int(rng.integers(1, 30))
            C = W * H * ch
            plane = int(rng.integers(0, ch))
            cap = (W // 4) * H
            flags = S.LAYOUT_PAPER2
            geo = dict(width=W, height=H, channels=ch, plane=plane)
        else:
            C = int(rng.integers(0, 200000))
            header = rng.random() < 0.7
            flags = S.HEADER_BE32 if header else 0
            cap = C // 8 - (4 if header else 0)
            if header and C < 32:
                cap = -1
            geo = {}
        over = rng.random() < 0.08
        if cap < 0:
            m = 0
        else:
            m = cap + 1 if over else int(rng.integers(0, cap + 1))
        cover = rng.integers(0, 256, C, dtype=np.uint8)
        msg = rng.integers(0, 256, m, dtype=np.uint8)
        inplace = rng.random() < 0.25
        off = int(rng.integers(0, 16))
        soff = off if (inplace or rng.random() < 0.5) else int(rng.integers(0, 16))
        cbuf = torch.empty(C + 32, dtype=torch.uint8, device="cuda")
        cv = cbuf[off:off + C]
        cv.copy_(torch.from_numpy(cover).cuda())
        if inplace:
            sv = cv
        else:
            sbuf = torch.full((C + 32,), 0x5A, dtype=torch.uint8, device="cuda")
            sv = sbuf[soff:soff + C]
            keep.append(sbuf)
        mv = torch.from_numpy(msg).cuda() if m else torch.empty(0, dtype=torch.uint8, device="cuda")
        ov = torch.full((m + 8,), 0xEE, dtype=torch.uint8, device="cuda")
        keep += [cbuf, mv, ov]
        recs.append(dict(cover=cv, stego=sv, msg=mv, cover_bytes=C, msg_bytes=m, flags=flags,
                         **geo))
        exts.append(dict(cover=sv, msg=ov, cover_bytes=C, msg_bytes=m + 8, msg_len=m,
                         flags=flags, **geo))
        if paper:
            st, want = O.paper2_embed(cover, W, H, ch, plane, msg)
        else:
            st, want = O.stream1_embed(cover, msg, header=bool(flags & S.HEADER_BE32))
            if st == oracle.OK and C == 0:
                want = cover
        checks.append((st, want, cover, msg, sv, ov, inplace))
    return recs, exts, checks, keep


@pytest.mark.parametrize("tile", [4096, 65536])
def test_random_batches(S, O, tile):
    rng = np.random.default_rng(7 + tile)
    for b in range(3):
        recs, exts, checks, keep = _batch(S, O, rng, 150)
        n = len(recs)
        d = S.descs_to_device(S.pack_descs(recs))
        res = S.new_result(n=n)
        ws = torch.empty(S.stego_batched_workspace_bytes(n), dtype=torch.uint8, device="cuda")
        S.stego_embed_batched(d, n, res, S.FUSE_STATS, ws, tune=(0, 0, 0, tile))
        rr = S.read_result(res)
        ok = []
        for i, (st, want, cover, msg, sv, ov, inplace) in enumerate(checks):
            assert rr[i]["status"] == st, (b, i, rr[i], st)
            got = sv.cpu().numpy()
            if st != oracle.OK:
                # nothing written: the cover in place, the 0x5A fill otherwise
                assert np.array_equal(got, cover) if inplace else np.all(got == 0x5A), (b, i)
                continue
            assert np.array_equal(got, want), (b, i, recs[i]["flags"], len(cover), len(msg))
            assert (rr[i]["changed"], rr[i]["sse"]) == O.changed_bytes(cover, want), (b, i)
            ok.append(i)
        # extract only what was embedded
        ex = [exts[i] for i in ok]
        if not ex:
            continue
        d2 = S.descs_to_device(S.pack_descs(ex))
        res2 = S.new_result(n=len(ex))
        ws2 = torch.empty(S.stego_batched_workspace_bytes(len(ex)), dtype=torch.uint8,
                          device="cuda")
        S.stego_extract_batched(d2, len(ex), res2, 0, ws2, tune=(0, 0, 0, tile))
        rr2 = S.read_result(res2)
        for j, i in enumerate(ok):
            st, want, cover, msg, sv, ov, inplace = checks[i]
            assert rr2[j]["status"] == 0 and rr2[j]["msg_bytes"] == len(msg), (b, i, rr2[j])
            out = ov.cpu().numpy()
            assert np.array_equal(out[:len(msg)], msg) and np.all(out[len(msg):] == 0xEE), (b, i)
