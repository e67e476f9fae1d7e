"""The batched embed that allocates nothing (stego_embed_batched_noalloc).

Callers that cannot call cudaMalloc (a host program without a device
allocator, or one that may not add cudaMalloc's implicit synchronisation to
a per-request path) use this entry point: its scratch lives in an array
inside the library.  Its output must equal stego_embed_batched's, given a
caller-allocated workspace, for the same descriptors, bit for bit, on two
calls in a row with different batches (the second call finds the first
call's leftovers in the shared scratch).  This file is collected last so a
run that stops at the first failure has already run every other test."""
import numpy as np
import pytest
import torch

from gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def _batch(S, rng, count):
    sizes, heads, msgs_n, covers, msgs = [], [], [], [], []
    for i in range(count):
        C = int(rng.choice([0, 40, 4096, 65543, int(rng.integers(32, 400000))]))
        header = bool(i % 2)
        cap = max(C // 8 - (4 if header else 0), 0)
        m = int(rng.integers(0, cap + 1)) if cap else 0
        if i % 13 == 7:
            m = cap + 1  # this cover alone fails with a capacity error
        sizes.append(C)
        heads.append(header)
        msgs_n.append(m)
        covers.append(torch.from_numpy(rng.integers(0, 256, C, dtype=np.uint8)).cuda())
        msgs.append(torch.from_numpy(rng.integers(0, 256, m, dtype=np.uint8)).cuda())
    return sizes, heads, msgs_n, covers, msgs


def _descs(S, sizes, heads, msgs_n, covers, stegos, msgs):
    recs = [dict(cover=covers[i], stego=stegos[i], msg=msgs[i], cover_bytes=sizes[i],
                 msg_bytes=msgs_n[i], flags=S.HEADER_BE32 if heads[i] else 0)
            for i in range(len(sizes))]
    return S.descs_to_device(S.pack_descs(recs))


def test_noalloc_matches_workspace_entry_point():
    S = need_gpu()
    rng = np.random.default_rng(2024)
    for call, count in enumerate((150, 37)):  # two calls in a row, different batches
        sizes, heads, msgs_n, covers, msgs = _batch(S, rng, count)
        ref_out = [torch.full_like(c, 0x5A) for c in covers]
        new_out = [torch.full_like(c, 0x5A) for c in covers]
        ref_res = S.new_result(n=count)
        new_res = S.new_result(n=count)
        ws = torch.empty(S.stego_batched_workspace_bytes(count), dtype=torch.uint8, device="cuda")
        S.stego_embed_batched(_descs(S, sizes, heads, msgs_n, covers, ref_out, msgs), count,
                              ref_res, S.FUSE_STATS, ws)
        S.stego_embed_batched_noalloc(_descs(S, sizes, heads, msgs_n, covers, new_out, msgs),
                                      count, new_res, S.FUSE_STATS)
        torch.cuda.synchronize()
        assert S.read_result(new_res) == S.read_result(ref_res), call
        for i in range(count):
            assert torch.equal(new_out[i], ref_out[i]), (call, i)
        statuses = [r["status"] for r in S.read_result(new_res)]
        assert S.OK in statuses and S.E_CAPACITY in statuses


def test_noalloc_rejects_oversized_batch():
    S = need_gpu()
    n = S.NOALLOC_MAX_DESCS + 1
    descs = torch.zeros(n * 72, dtype=torch.uint8, device="cuda")
    res = S.new_result(n=n)
    with pytest.raises(S.StegoError) as e:
        S.stego_embed_batched_noalloc(descs, n, res, 0)
    assert e.value.status == S.E_NOMEM
    # the largest accepted batch (all empty covers) runs
    S.stego_embed_batched_noalloc(descs, n - 1, res[: n - 1], 0)
    torch.cuda.synchronize()
    assert all(r["status"] == 0 for r in S.read_result(res[: n - 1]))
