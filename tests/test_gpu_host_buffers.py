"""Kernels working directly on pinned host buffers (zero-copy over the
CPU-GPU link): same bytes as the oracle and as the device-memory path."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    return need_gpu()


def _pinned(a):
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory()


def test_pinned_pointers_are_reported_accessible(S):
    t = torch.empty(4096, dtype=torch.uint8).pin_memory()
    kind, acc = S.stego_pointer_kind(t.data_ptr())
    assert kind == S.MEM_PINNED and acc
    d = torch.empty(4096, dtype=torch.uint8, device="cuda")
    assert S.stego_pointer_kind(d.data_ptr()) == (S.MEM_DEVICE, True)


@pytest.mark.parametrize("C", [4097, 1 << 20, 3 * 65536 + 24])
def test_embed_extract_on_host_buffers(S, C):
    O = oracle.load()
    rng = np.random.default_rng(C)
    cover = rng.integers(0, 256, C, dtype=np.uint8)
    msg = rng.integers(0, 256, C // 8 - 4, dtype=np.uint8)
    st, want = O.stream1_embed(cover, msg, header=True)
    assert st == 0
    c_h, m_h = _pinned(cover), _pinned(msg)
    s_h = torch.full((C,), 0x5A, dtype=torch.uint8).pin_memory()
    res = S.new_result()
    S.stego_embed(c_h, s_h, m_h, S.HEADER_BE32 | S.FUSE_STATS, res)
    torch.cuda.synchronize()
    assert np.array_equal(s_h.numpy(), want)
    r = S.read_result(res)
    assert (r["changed"], r["sse"]) == O.changed_bytes(cover, want)
    out_h = torch.full((msg.size + 5,), 0xEE, dtype=torch.uint8).pin_memory()
    res2 = S.new_result()
    S.stego_extract(s_h, out_h, 0, S.HEADER_BE32, res2)
    torch.cuda.synchronize()
    assert np.array_equal(out_h.numpy()[: msg.size], msg)
    assert np.all(out_h.numpy()[msg.size:] == 0xEE)
    # mixed: device cover, host stego
    s2 = torch.zeros(C, dtype=torch.uint8).pin_memory()
    S.stego_embed(c_h.cuda(), s2, m_h.cuda(), S.HEADER_BE32)
    torch.cuda.synchronize()
    assert np.array_equal(s2.numpy(), want)


def test_batched_descriptors_pointing_at_host_buffers(S):
    O = oracle.load()
    rng = np.random.default_rng(5)
    sizes = [5000, 65536, 123457, 40]
    covers = [_pinned(rng.integers(0, 256, c, dtype=np.uint8)) for c in sizes]
    msgs = [_pinned(rng.integers(0, 256, c // 8 - 4, dtype=np.uint8)) for c in sizes]
    stegos = [torch.empty(c, dtype=torch.uint8).pin_memory() for c in sizes]
    recs = [dict(cover=covers[i], stego=stegos[i], msg=msgs[i], cover_bytes=sizes[i],
                 msg_bytes=msgs[i].numel(), flags=S.HEADER_BE32) for i in range(len(sizes))]
    descs = S.descs_to_device(S.pack_descs(recs))
    res = S.new_result(n=len(sizes))
    ws = torch.empty(S.stego_batched_workspace_bytes(len(sizes)), dtype=torch.uint8, device="cuda")
    S.stego_embed_batched(descs, len(sizes), res, S.FUSE_STATS, ws)
    torch.cuda.synchronize()
    for i in range(len(sizes)):
        st, want = O.stream1_embed(covers[i].numpy(), msgs[i].numpy(), header=True)
        assert st == 0 and np.array_equal(stegos[i].numpy(), want), i
