"""Seeded random combinations of every single-cover option against the CPU
oracle, byte for byte: layout, bits per byte, one plane or all bytes,
channels, geometry, header or raw, message length, in place or not, and the
offsets of cover, stego and message buffers from a 16-byte boundary (which
select the vector, head-and-vector and byte kernels).  Canary bytes around
every output catch stray writes."""
import numpy as np
import pytest

import oracle
from gpu_util import Guarded, need_gpu

pytestmark = pytest.mark.gpu

CASES = 1000


@pytest.fixture(scope="module")
def S():
    return need_gpu()


@pytest.fixture(scope="module")
def O():
    return oracle.load()


def _case(rng):
    layout = rng.choice(["stream", "stream", "stream", "paper"])
    ch = int(rng.choice([1, 2, 3, 4]))
    W = int(rng.integers(1, 200))
    H = int(rng.integers(1, 40))
    if rng.random() < 0.3:
        W = 16 * int(rng.integers(1, 12))  # rows of whole vectors (unit kernels)
    plane = int(rng.integers(0, ch))
    k = int(rng.integers(1, 5)) if layout == "stream" else 1
    plane_only = layout == "stream" and rng.random() < 0.5
    header = layout == "stream" and rng.random() < 0.7
    inplace = rng.random() < 0.3
    same = rng.random() < 0.5
    oc = int(rng.integers(0, 16))
    os_ = oc if (inplace or same) else int(rng.integers(0, 16))
    om = int(rng.integers(0, 16))
    return dict(layout=layout, ch=ch, W=W, H=H, plane=plane, k=k, plane_only=plane_only,
                header=header, inplace=inplace, offs=(oc, os_, om))


def test_random_combinations(S, O):
    rng = np.random.default_rng(20261203)
    done = 0
    for n in range(CASES):
        c = _case(rng)
        C = c["W"] * c["H"] * c["ch"]
        cover = rng.integers(0, 256, C, dtype=np.uint8)
        geom = (c["W"], c["H"], c["ch"], c["plane"])
        if c["layout"] == "paper":
            flags = S.LAYOUT_PAPER2
            cap = (c["W"] // 4) * c["H"]
        else:
            flags = S.BITS(c["k"]) | (S.HEADER_BE32 if c["header"] else 0) | \
                (S.PLANE_ONLY if c["plane_only"] else 0)
            try:
                cap = S.stego_capacity(C, flags, geom=geom if c["plane_only"] else None)
            except S.StegoError:
                continue
        if cap <= 0 and c["header"]:
            continue
        m = int(rng.integers(0, max(cap, 0) + 1))
        msg = rng.integers(0, 256, m, dtype=np.uint8)
        g = geom if (c["layout"] == "paper" or c["plane_only"]) else None
        if c["layout"] == "paper":
            st, want = O.paper2_embed(cover, *geom, msg)
        else:
            st, want = O.streamk_embed(cover, msg, c["k"], header=c["header"], geom=g)
        if st != oracle.OK:
            continue
        oc, os_, om = c["offs"]
        gc = Guarded(C, oc, cover)
        gm = Guarded(m, om, msg)
        gs = gc if c["inplace"] else Guarded(C, os_, 0x5A)
        res = S.new_result()
        S.stego_embed(gc.view, gs.view, gm.view, flags | S.FUSE_STATS, res, geom=g)
        got = gs.host()
        assert np.array_equal(got, want), (n, c, m)
        assert gs.canaries_intact() and gc.canaries_intact() and gm.canaries_intact(), (n, c)
        r = S.read_result(res)
        assert r["status"] == 0 and r["msg_bytes"] == m, (n, c, r)
        assert (r["changed"], r["sse"]) == O.changed_bytes(cover, want), (n, c)
        # extraction from a stego at the stego offset into a stale buffer
        cap_out = m + 3
        gx = Guarded(want.size, os_, want)
        go = Guarded(cap_out, (om + 5) % 16, 0xEE)
        res2 = S.new_result()
        S.stego_extract(gx.view, go.view, m, flags, res2, geom=g)
        r2 = S.read_result(res2)
        assert r2["status"] == 0 and r2["msg_bytes"] == m, (n, c, r2)
        out = go.host()
        assert np.array_equal(out[:m], msg) and np.all(out[m:] == 0xEE), (n, c)
        assert go.canaries_intact(), (n, c)
        done += 1
    assert done > CASES // 2
