"""The C-ABI library builds, loads and exports every function that
include/stego.h declares; host-only entry points (no device work) behave as
documented.  Runs without a GPU."""
import ctypes
import os
import re

import pytest

from paper_0912_0947_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    try:
        B.nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available")
    return B.build()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "stego.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(stego_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("stego_embed", "stego_extract", "stego_embed_batched", "stego_extract_batched",
              "stego_changed_bytes", "stego_capacity", "stego_strerror",
              "stego_batched_workspace_bytes"):
        assert n in names


def test_library_exports_every_declared_function(built):
    lib = ctypes.CDLL(built)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_entry_points(built):
    import paper_0912_0947_gb300 as S
    assert S.stego_version() >= 10000
    assert S.strerror(S.E_BAD_HEADER) == "bad or missing length header"
    # capacities: floor(C/8) - 4 with the header, floor(C/8) raw, floor(W/4)*H
    assert S.stego_capacity(201326592, S.HEADER_BE32) == 25165820
    assert S.stego_capacity(786432, S.HEADER_BE32) == 98300
    assert S.stego_capacity(31, S.HEADER_BE32) == 0
    assert S.stego_capacity(41, 0) == 5
    assert S.stego_capacity(1024, S.LAYOUT_PAPER2, (1024, 1, 1, 0)) == 256
    assert S.stego_capacity(7 * 5 * 3, S.LAYOUT_PAPER2, (7, 5, 3, 2)) == 5
    with pytest.raises(S.StegoError):
        S.stego_capacity(100, S.LAYOUT_PAPER2, (7, 5, 3, 3))  # plane >= channels
    with pytest.raises(S.StegoError):
        S.stego_capacity(100, S.LAYOUT_PAPER2, (7, 5, 3, 0))  # size mismatch
    assert S.stego_batched_workspace_bytes(0) >= 64
    assert S.stego_batched_workspace_bytes(4096) >= 64 + 8 * 4097 + 32 * 4096


def test_tune_validation(built):
    import paper_0912_0947_gb300 as S
    old = S.stego_get_tune(S.OP_EMBED)
    with pytest.raises(S.StegoError):
        S.stego_set_tune(S.OP_EMBED, (100, 4, 0, 0))   # not a multiple of 32
    with pytest.raises(S.StegoError):
        S.stego_set_tune(S.OP_EMBED, (256, 3, 0, 0))   # vec not in {1,2,4,8}
    with pytest.raises(S.StegoError):
        S.stego_set_tune(S.OP_EMBED_BATCHED, (256, 4, 0, 5000))  # tile not 4 KiB multiple
    with pytest.raises(S.StegoError):
        S.stego_set_tune(9, (256, 4, 0, 0))
    S.stego_set_tune(S.OP_EMBED, (128, 2, 3, 0))
    t = S.stego_get_tune(S.OP_EMBED)
    assert (t.threads, t.vec_per_thread, t.ctas_per_sm) == (128, 2, 3)
    # single-cover calls install tile_bytes as given (0 = register kernels),
    # batched calls keep their tile when given 0
    S.stego_set_tune(S.OP_EMBED, (256, 4, 0, 65536))
    assert S.stego_get_tune(S.OP_EMBED).tile_bytes == 65536
    S.stego_set_tune(S.OP_EMBED, (256, 4, 0, 0))
    assert S.stego_get_tune(S.OP_EMBED).tile_bytes == 0
    oldb = S.stego_get_tune(S.OP_EXTRACT_BATCHED)
    S.stego_set_tune(S.OP_EXTRACT_BATCHED, (256, 4, 0, 0))
    assert S.stego_get_tune(S.OP_EXTRACT_BATCHED).tile_bytes == oldb.tile_bytes
    S.stego_set_tune(S.OP_EMBED, old)


def test_struct_sizes_match_header():
    import paper_0912_0947_gb300 as S
    assert S.DESC_DTYPE.itemsize == 72
    assert ctypes.sizeof(S.Geom) == 16 and ctypes.sizeof(S.Tune) == 16


def test_binding_refuses_cpu_tensors(built):
    import torch
    import paper_0912_0947_gb300 as S
    c = torch.zeros(64, dtype=torch.uint8)
    with pytest.raises(ValueError):
        S.stego_embed(c, c.clone(), torch.zeros(1, dtype=torch.uint8), S.HEADER_BE32)


def test_product_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_0912_0947_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "stego_oracle" not in text, f


def test_header_compiles_as_c():
    """include/stego.h is plain C: the C example that uses it compiles with
    gcc (syntax only, no GPU needed)."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not gcc or not os.path.exists(nvcc):
        pytest.skip("gcc or the CUDA toolkit not available")
    cuda = os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    here = os.path.dirname(os.path.abspath(__file__))
    r = subprocess.run([gcc, "-std=c11", "-Wall", "-Wextra", "-Werror", "-fsyntax-only",
                        os.path.join(here, "c", "abi_roundtrip.c"),
                        "-I" + os.path.join(os.path.dirname(here), "include"),
                        "-I" + os.path.join(cuda, "include")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_capacity_is_the_oracles_boundary(built):
    """stego_capacity (host code of the library) for every layout, header
    choice, bits per byte and plane against the oracle: a message of the
    reported capacity embeds, one byte more is refused."""
    import numpy as np
    import oracle
    import paper_0912_0947_gb300 as S
    O = oracle.load()
    rng = np.random.default_rng(77)
    geoms = [(7, 5, 3, 2), (16, 3, 1, 0), (33, 2, 4, 1), (5, 9, 3, 0), (64, 1, 3, 1)]
    for W, H, ch, plane in geoms:
        C = W * H * ch
        cover = rng.integers(0, 256, C, dtype=np.uint8)
        for k in (1, 2, 3, 4):
            for header in (True, False):
                for plane_only in (False, True):
                    flags = S.BITS(k) | (S.HEADER_BE32 if header else 0) | \
                        (S.PLANE_ONLY if plane_only else 0)
                    g = (W, H, ch, plane) if plane_only else None
                    cap = S.stego_capacity(C, flags, geom=g)
                    ok = rng.integers(0, 256, cap, dtype=np.uint8)
                    over = rng.integers(0, 256, cap + 1, dtype=np.uint8)
                    st, _ = O.streamk_embed(cover, ok, k, header=header, geom=g)
                    assert st == oracle.OK, (W, H, ch, plane, k, header, plane_only, cap)
                    st, _ = O.streamk_embed(cover, over, k, header=header, geom=g)
                    assert st != oracle.OK, (W, H, ch, plane, k, header, plane_only, cap)
        cap = S.stego_capacity(C, S.LAYOUT_PAPER2, (W, H, ch, plane))
        assert cap == O.paper2_capacity(W, H)
        st, _ = O.paper2_embed(cover, W, H, ch, plane, rng.integers(0, 256, cap, dtype=np.uint8))
        assert st == oracle.OK
        st, _ = O.paper2_embed(cover, W, H, ch, plane,
                               rng.integers(0, 256, cap + 1, dtype=np.uint8))
        assert st != oracle.OK


def test_host_job_packing():
    """stego_host_job records (80 bytes) packed from CPU tensors: pointers,
    sizes, flags and geometry land in their fields; None is a null pointer."""
    import numpy as np
    import torch

    import paper_0912_0947_gb300 as S
    c = torch.zeros(100, dtype=torch.uint8)
    m = torch.zeros(7, dtype=torch.uint8)
    a = S.Pipeline.jobs([dict(cover=c, stego=c, msg=m, readback=None, cover_bytes=100,
                              msg_bytes=7, msg_len=3, flags=S.LAYOUT_PAPER2, width=10,
                              height=5, channels=2, plane=1)])
    assert a.dtype.itemsize == 80
    r = a[0]
    assert r["cover"] == r["stego"] == c.data_ptr() and r["msg"] == m.data_ptr()
    assert r["readback"] == 0
    assert (r["cover_bytes"], r["msg_bytes"], r["msg_len"]) == (100, 7, 3)
    assert (r["flags"], r["width"], r["height"], r["channels"], r["plane"]) == (1, 10, 5, 2, 1)
    raw = a.view(np.uint64)  # the pointer and size words in C order
    assert int(raw[0]) == c.data_ptr() and int(raw[4]) == 100
    with pytest.raises(TypeError):  # device tensors are not host buffers
        S.Pipeline.jobs([dict(cover=torch.zeros(4, dtype=torch.uint8, device="meta"))])
