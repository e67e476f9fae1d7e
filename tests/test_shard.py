"""Several GPUs, host side (CPU): the byte-volume partition of a batch
(stego_partition) and the sharded runner's gather, with two gloo ranks on
the CPU.  The per-cover work in the gloo test is the oracle's embed (there
is no GPU here); the point is the host logic: every cover on exactly one
rank, the ranks within one cover's bytes of each other, and the gathered
per-cover results equal to one process's over the whole batch."""
import json
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import paper_0912_0947_gb300 as S
from paper_0912_0947_gb300 import shard, synth


def test_partition_balanced_within_one_cover():
    items = synth.uneven_batch(4096)
    sizes = np.array([it.cover_bytes for it in items], dtype=np.uint64)
    for world in (1, 2, 3, 4, 7, 8):
        rank_of, rank_bytes = S.stego_partition(sizes, world)
        assert rank_of.shape == (4096,) and rank_of.max() < world
        loads = np.bincount(rank_of, weights=sizes.astype(np.float64), minlength=world)
        assert np.array_equal(loads.astype(np.uint64), rank_bytes)
        assert int(rank_bytes.sum()) == int(sizes.sum())
        assert int(rank_bytes.max() - rank_bytes.min()) <= int(sizes.max())
        # deterministic: the same split every time
        assert np.array_equal(S.stego_partition(sizes, world)[0], rank_of)
        parts = [shard.my_covers(sizes, r, world) for r in range(world)]
        assert sorted(np.concatenate(parts).tolist()) == list(range(4096))


def test_partition_small_cases():
    # largest first, each to the least-loaded rank (ties to the lower rank)
    rank_of, rank_bytes = S.stego_partition([5, 9, 1, 7, 3, 3], 2)
    assert rank_of.tolist() == [1, 0, 1, 1, 0, 0] and rank_bytes.tolist() == [15, 13]
    rank_of, rank_bytes = S.stego_partition([], 3)
    assert rank_of.size == 0 and rank_bytes.tolist() == [0, 0, 0]
    rank_of, rank_bytes = S.stego_partition([4, 4], 5)  # more ranks than covers
    assert rank_of.tolist() == [0, 1] and rank_bytes.tolist() == [4, 4, 0, 0, 0]
    for world in (0, (1 << 16) + 1):
        with pytest.raises(S.StegoError) as e:
            S.stego_partition([1, 2], world)
        assert e.value.status == S.E_INVAL


def _batch():
    items = synth.uneven_batch(48, lo=16, hi=300)
    rng = np.random.default_rng(5)
    covers = [rng.integers(0, 256, it.cover_bytes, dtype=np.uint8) for it in items]
    msgs = [rng.integers(0, 256, it.msg_bytes, dtype=np.uint8) for it in items]
    return [it.cover_bytes for it in items], covers, msgs


def _compute(idx):
    import oracle
    O = oracle.load()
    _, covers, msgs = _batch()
    out = []
    for i in idx:
        st, w = O.stream1_embed(covers[i], msgs[i], header=True)
        ch, sse = O.changed_bytes(covers[i], w)
        out.append({"status": st, "changed": ch, "sse": sse, "sum": int(w.sum(dtype=np.uint64))})
    return out


def _rank_main(rank, world, port, path):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    sizes, _, _ = _batch()
    got = shard.run_sharded(sizes, rank, world, _compute)
    mine = shard.my_covers(sizes, rank, world).tolist()
    if rank == 0:
        with open(path, "w") as f:
            json.dump({"results": got}, f)
    with open(path + ".rank%d" % rank, "w") as f:
        json.dump(mine, f)
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_sharded_two_gloo_ranks_equal_one_process(tmp_path):
    path = str(tmp_path / "gathered.json")
    mp.spawn(_rank_main, args=(2, _free_port(), path), nprocs=2, join=True)
    with open(path) as f:
        got = json.load(f)["results"]
    sizes, _, _ = _batch()
    want = _compute(range(len(sizes)))
    assert got == want
    # the two ranks' shares are disjoint, cover everything and balance bytes
    shares = [json.load(open(path + ".rank%d" % r)) for r in range(2)]
    assert sorted(shares[0] + shares[1]) == list(range(len(sizes)))
    b = [sum(sizes[i] for i in sh) for sh in shares]
    assert abs(b[0] - b[1]) <= max(sizes)
    # one process, no collective: the same results
    assert shard.run_sharded(sizes, 0, 1, _compute) == want


# ---------------------------------------------------------------- one cover

def test_cover_slices_tile_the_cover():
    for C in (0, 5, 16, 100, 4097, (1 << 20) + 3):
        for world in range(1, 10):
            sl = shard.cover_slices(C, world)
            assert len(sl) == world and sl[0][0] == 0 and sl[-1][1] == C
            assert all(a % 16 == 0 and a <= b for a, b in sl)
            assert all(sl[i][1] == sl[i + 1][0] for i in range(world - 1))
            sizes = [b - a for a, b in sl]
            assert max(sizes) - min(sizes) <= 16 + 15
    with pytest.raises(ValueError):
        shard.cover_slices(10, 0)


@pytest.mark.parametrize("header", [True, False])
def test_slice_message_ranges_partition_the_message(header):
    for C in (32, 48, 1000, 4097, 65536 + 40):
        cap = S.stego_capacity(C, S.HEADER_BE32 if header else 0)
        for m in sorted({0, min(1, cap), cap // 2, cap}):
            for world in (1, 2, 3, 7):
                got = []
                for c0, c1 in shard.cover_slices(C, world):
                    for kind, a, b, lo, hi in shard.slice_pieces(c0, c1, m, header):
                        assert c0 <= a < b <= c1 and a % 8 == 0
                        if kind == "msg":
                            got.append((lo, hi))
                            assert 8 * (lo + (4 if header else 0)) == a or lo == hi
                        else:
                            assert header and b <= 32 and (lo, hi) == (a // 8, b // 8)
                lo_hi = [r for r in got if r[1] > r[0]]
                assert all(lo_hi[i][1] == lo_hi[i + 1][0] for i in range(len(lo_hi) - 1))
                if m:
                    assert (lo_hi[0][0], lo_hi[-1][1]) == (0, m)
                else:
                    assert lo_hi == []


def _oracle_slice(O, cover, msg, c0, c1, m, header):
    """One slice through its pieces, each a raw oracle embed."""
    parts, ch, ss = [], 0, 0
    for kind, a, b, lo, hi in shard.slice_pieces(c0, c1, m, header):
        src = (np.frombuffer(shard.header_bytes(m), np.uint8)[lo:hi] if kind == "header"
               else msg[lo:hi])
        st, w = O.stream1_embed(cover[a:b], src, header=False)
        assert st == 0
        parts.append(w)
        c, s_ = O.changed_bytes(cover[a:b], w)
        ch, ss = ch + c, ss + s_
    return (np.concatenate(parts) if parts else np.zeros(0, np.uint8)), ch, ss


@pytest.mark.parametrize("header", [True, False])
def test_slices_through_raw_pieces_equal_one_embed(header):
    """The slice plan executed with the oracle's raw embed reproduces the
    oracle's embed of the whole stream, stats included."""
    import oracle
    O = oracle.load()
    rng = np.random.default_rng(77 + header)
    for C in (32, 40, 1000, 4101, 3 * 4096 + 16 + 7):
        cover = rng.integers(0, 256, C, dtype=np.uint8)
        cap = S.stego_capacity(C, S.HEADER_BE32 if header else 0)
        for m in sorted({0, min(1, cap), cap // 3, cap}):
            msg = rng.integers(0, 256, m, dtype=np.uint8)
            st, want = O.stream1_embed(cover, msg, header=header)
            assert st == 0
            for world in (1, 2, 3, 5, 8):
                got, ch, ss = [], 0, 0
                for c0, c1 in shard.cover_slices(C, world):
                    w, c, s_ = _oracle_slice(O, cover, msg, c0, c1, m, header)
                    assert w.size == c1 - c0
                    got.append(w)
                    ch, ss = ch + c, ss + s_
                assert np.array_equal(np.concatenate(got), want), (C, m, world)
                assert (ch, ss) == O.changed_bytes(cover, want)


def _split_rank(rank, world, port, path):
    import torch.distributed as dist
    import oracle
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    O = oracle.load()
    rng = np.random.default_rng(123)
    C = 20000 + 7
    cover = rng.integers(0, 256, C, dtype=np.uint8)
    m = S.stego_capacity(C, S.HEADER_BE32) - 5
    msg = rng.integers(0, 256, m, dtype=np.uint8)
    c0, c1 = shard.cover_slices(C, world)[rank]
    w, ch, ss = _oracle_slice(O, cover, msg, c0, c1, m, True)
    got = shard.gather_results(np.array([rank]), [(w.tobytes(), ch, ss)], world)
    if rank == 0:
        st, want = O.stream1_embed(cover, msg, header=True)
        ok = (b"".join(g[0] for g in got) == want.tobytes() and
              (sum(g[1] for g in got), sum(g[2] for g in got)) == O.changed_bytes(cover, want))
        with open(path, "w") as f:
            json.dump({"ok": bool(ok), "ranks": len(got)}, f)
    dist.barrier()
    dist.destroy_process_group()


def test_single_cover_split_two_gloo_ranks(tmp_path):
    path = str(tmp_path / "split.json")
    mp.spawn(_split_rank, args=(2, _free_port(), path), nprocs=2, join=True)
    with open(path) as f:
        assert json.load(f) == {"ok": True, "ranks": 2}
