"""The batched embed that allocates nothing (stego_embed_batched_noalloc).

Callers that cannot call cudaMalloc (a host program without a device
allocator, or one that may not add cudaMalloc's implicit synchronisation to
a per-request path) use this entry point: its scratch lives in an array
inside the library.  Its output must equal stego_embed_batched's, given a
caller-allocated workspace, for the same descriptors, bit for bit, and the
oracle's, on two calls in a row with different batches (the second call
finds the first call's leftovers in the shared scratch).  Both batches mix
one-bit stream covers with paper-layout covers (Sections VI/VII), whose
tiles use their own scratch fields, in place and out of place, with rows of
whole vectors and rows that are not.  This file is collected last so a run
that stops at the first failure has already run every other test."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import need_gpu

pytestmark = pytest.mark.gpu

# paper-layout covers of each batch: (width, height, channels, plane, in place)
PAPER_GEOMS = [
    [(1920, 9, 3, 0, False), (1920, 6, 3, 0, True), (33, 7, 3, 2, False), (64, 16, 4, 3, True),
     (1024, 3, 1, 0, False)],
    [(160, 12, 1, 0, True), (4000, 6, 4, 2, False), (9, 4, 3, 1, True), (512, 20, 3, 0, False)],
]


def _batch(S, rng, count, paper):
    """Per cover: (flags, geometry dict, cover bytes, message bytes, in place,
    cover array, message array)."""
    items = []
    for i in range(count):
        C = int(rng.choice([0, 40, 4096, 65543, int(rng.integers(32, 400000))]))
        header = bool(i % 2)
        cap = max(C // 8 - (4 if header else 0), 0)
        m = int(rng.integers(0, cap + 1)) if cap else 0
        if i % 13 == 7:
            m = cap + 1  # this cover alone fails with a capacity error
        items.append(dict(flags=S.HEADER_BE32 if header else 0, geo={}, C=C, m=m,
                          inplace=False, cover=rng.integers(0, 256, C, dtype=np.uint8),
                          msg=rng.integers(0, 256, m, dtype=np.uint8)))
    for W, H, ch, pl, inplace in paper:
        C = W * H * ch
        m = int(rng.integers(1, (W // 4) * H + 1))
        items.append(dict(flags=S.LAYOUT_PAPER2,
                          geo=dict(width=W, height=H, channels=ch, plane=pl), C=C, m=m,
                          inplace=inplace, cover=rng.integers(0, 256, C, dtype=np.uint8),
                          msg=rng.integers(0, 256, m, dtype=np.uint8)))
    return items


def _run(S, items, noalloc):
    """Embeds the batch with one entry point; returns outputs and results."""
    n = len(items)
    outs, recs, keep = [], [], []
    for it in items:
        c = torch.from_numpy(it["cover"]).cuda()
        o = c if it["inplace"] else torch.full_like(c, 0x5A)
        msg = torch.from_numpy(it["msg"]).cuda()
        keep += [c, msg]
        outs.append(o)
        recs.append(dict(cover=c, stego=o, msg=msg, cover_bytes=it["C"], msg_bytes=it["m"],
                         flags=it["flags"], **it["geo"]))
    descs = S.descs_to_device(S.pack_descs(recs))
    res = S.new_result(n=n)
    if noalloc:
        S.stego_embed_batched_noalloc(descs, n, res, S.FUSE_STATS)
    else:
        ws = torch.empty(S.stego_batched_workspace_bytes(n), dtype=torch.uint8, device="cuda")
        S.stego_embed_batched(descs, n, res, S.FUSE_STATS, ws)
    torch.cuda.synchronize()
    return outs, S.read_result(res)


def test_noalloc_matches_workspace_entry_point_and_oracle():
    S = need_gpu()
    O = oracle.load()
    rng = np.random.default_rng(2024)
    for call, count in enumerate((150, 37)):  # two calls in a row, different batches
        items = _batch(S, rng, count, PAPER_GEOMS[call])
        ref_out, ref_res = _run(S, items, noalloc=False)
        new_out, new_res = _run(S, items, noalloc=True)
        assert new_res == ref_res, call
        for i, it in enumerate(items):
            assert torch.equal(new_out[i], ref_out[i]), (call, i)
            if it["flags"] == S.LAYOUT_PAPER2:
                g = it["geo"]
                st, want = O.paper2_embed(it["cover"], g["width"], g["height"], g["channels"],
                                          g["plane"], it["msg"])
            else:
                st, want = O.stream1_embed(it["cover"], it["msg"],
                                           header=bool(it["flags"] & S.HEADER_BE32))
            r = new_res[i]
            assert r["status"] == st, (call, i)
            if st != 0:
                assert r["msg_bytes"] == 0
                assert bool((new_out[i] == 0x5A).all()), (call, i)  # not written
                continue
            assert np.array_equal(new_out[i].cpu().numpy(), want), (call, i)
            assert (r["changed"], r["sse"]) == O.changed_bytes(it["cover"], want), (call, i)
            assert r["msg_bytes"] == it["m"]
        statuses = [r["status"] for r in new_res]
        assert S.OK in statuses and S.E_CAPACITY in statuses


def test_noalloc_rejects_oversized_batch():
    S = need_gpu()
    n = S.NOALLOC_MAX_DESCS + 1
    descs = torch.zeros(n * 72, dtype=torch.uint8, device="cuda")
    res = S.new_result(n=n)
    with pytest.raises(S.StegoError) as e:
        S.stego_embed_batched_noalloc(descs, n, res, 0)
    assert e.value.status == S.E_NOMEM
    # bad flags are reported as such whatever the batch size
    with pytest.raises(S.StegoError) as e:
        S.stego_embed_batched_noalloc(descs, n, res, 0x4000)
    assert e.value.status == S.E_INVAL
    # the largest accepted batch (all empty covers) runs and rewrites every
    # result, each of which starts out as a sentinel
    res[:, 2] = 0xFFFF
    res[:, 3] = -1
    S.stego_embed_batched_noalloc(descs, n - 1, res[: n - 1], 0)
    torch.cuda.synchronize()
    rr = S.read_result(res)
    assert all(r["status"] == 0 and r["msg_bytes"] == 0 for r in rr[: n - 1])
    assert rr[n - 1]["status"] == -1 and rr[n - 1]["msg_bytes"] == 0xFFFF
