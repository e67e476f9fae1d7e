"""CPU oracle for LSB substitution steganography -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path
(``paper_0912_0947_gb300``) never imports it, and this package never imports
the product path: they share no code.

The arithmetic lives in ``stego_oracle.c`` (plain single-threaded C, built
with gcc into ``oracle/_build/libstego_oracle.so``).  This module only builds
that library and marshals numpy arrays into it.

Layouts (see the C file for the step-by-step reading of the paper):
  * ``stream1`` -- one bit per cover byte, memory order, stream
    ``BE32(8*m) || msg`` (header) or ``msg`` (raw), MSB first.
  * ``paper2`` -- Section VI / VII: one plane, two bits per byte, greedy row
    division with ``floor(W/4)`` bytes per row, pair i of ``B[j]`` at
    ``A[L*i + j]``.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "stego_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libstego_oracle.so")

OK = 0
E_INVAL = -1
E_CAPACITY = -2
E_BAD_HEADER = -3
E_MSG_TOO_SMALL = -4

# fill value of message buffers handed to the extractors (stale contents)
STALE = 0xCD

_u8p = ctypes.c_void_p
_u64 = ctypes.c_uint64
_u32 = ctypes.c_uint32


def build(src: str = _SRC, out: str = _LIB, quiet: bool = True) -> str:
    """Compile the oracle C file into a shared library (gcc, -O2)."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-Wall", "-Wextra", "-shared", "-fPIC",
           src, "-o", tmp]
    subprocess.run(cmd, check=True,
                   stdout=subprocess.DEVNULL if quiet else None)
    os.replace(tmp, out)
    return out


def _ptr(a):
    if a is None:
        return None
    return ctypes.c_void_p(a.ctypes.data)


class Oracle:
    """ctypes handle on one compiled oracle library."""

    def __init__(self, path: str = _LIB):
        lib = ctypes.CDLL(path)
        lib.oracle_stream1_embed.argtypes = [_u8p, _u8p, _u64, _u8p, _u64, ctypes.c_int]
        lib.oracle_stream1_embed.restype = ctypes.c_int
        lib.oracle_stream1_extract.argtypes = [_u8p, _u64, _u8p, _u64, ctypes.c_int,
                                               _u64, ctypes.POINTER(_u64)]
        lib.oracle_stream1_extract.restype = ctypes.c_int
        lib.oracle_paper2_capacity.argtypes = [_u32, _u32]
        lib.oracle_paper2_capacity.restype = _u64
        lib.oracle_paper2_embed.argtypes = [_u8p, _u8p, _u32, _u32, _u32, _u32, _u8p, _u64]
        lib.oracle_paper2_embed.restype = ctypes.c_int
        lib.oracle_paper2_extract.argtypes = [_u8p, _u32, _u32, _u32, _u32, _u8p, _u64, _u64]
        lib.oracle_paper2_extract.restype = ctypes.c_int
        lib.oracle_streamk_embed.argtypes = [_u8p, _u8p, _u64, _u32, ctypes.c_int, _u32, _u32,
                                             _u32, _u32, _u8p, _u64, ctypes.c_int]
        lib.oracle_streamk_embed.restype = ctypes.c_int
        lib.oracle_streamk_extract.argtypes = [_u8p, _u64, _u32, ctypes.c_int, _u32, _u32, _u32,
                                               _u32, _u8p, _u64, ctypes.c_int, _u64,
                                               ctypes.POINTER(_u64)]
        lib.oracle_streamk_extract.restype = ctypes.c_int
        lib.oracle_changed_bytes.argtypes = [_u8p, _u8p, _u64, ctypes.POINTER(_u64),
                                             ctypes.POINTER(_u64)]
        lib.oracle_changed_bytes.restype = None
        self.lib = lib
        self.path = path

    # -- stream1 ---------------------------------------------------------
    def stream1_embed(self, cover, msg, header=True, out=None):
        """Returns (status, stego).  On error stego is a copy of ``out``
        as passed (or of the cover when ``out`` is None) -- nothing written."""
        cover = np.ascontiguousarray(cover, dtype=np.uint8).reshape(-1)
        msg = np.ascontiguousarray(msg, dtype=np.uint8).reshape(-1)
        if out is None:
            out = np.zeros_like(cover)
        st = self.lib.oracle_stream1_embed(_ptr(cover), _ptr(out), cover.size,
                                           _ptr(msg), msg.size, int(bool(header)))
        return st, out

    def stream1_embed_inplace(self, buf, msg, header=True):
        buf = np.ascontiguousarray(buf, dtype=np.uint8).reshape(-1)
        msg = np.ascontiguousarray(msg, dtype=np.uint8).reshape(-1)
        st = self.lib.oracle_stream1_embed(_ptr(buf), _ptr(buf), buf.size,
                                           _ptr(msg), msg.size, int(bool(header)))
        return st, buf

    def stream1_extract(self, stego, cap=None, header=True, raw_len=0):
        """Returns (status, msg_bytes_array)."""
        stego = np.ascontiguousarray(stego, dtype=np.uint8).reshape(-1)
        if cap is None:
            cap = stego.size // 8
        # a buffer holding stale bytes, as a caller's reused buffer would
        msg = np.full(max(int(cap), 1), STALE, dtype=np.uint8)
        n = _u64(0)
        st = self.lib.oracle_stream1_extract(_ptr(stego), stego.size, _ptr(msg), int(cap),
                                             int(bool(header)), int(raw_len), ctypes.byref(n))
        return st, msg[: n.value].copy()

    # -- streamk: k bits per carrying byte, all bytes or one plane ---------
    def streamk_embed(self, cover, msg, k, header=True, geom=None, out=None):
        """geom=(W, H, channels, plane) selects one plane (plane_only)."""
        cover = np.ascontiguousarray(cover, dtype=np.uint8).reshape(-1)
        msg = np.ascontiguousarray(msg, dtype=np.uint8).reshape(-1)
        if out is None:
            out = np.zeros_like(cover)
        W, H, C, p = geom if geom is not None else (0, 0, 0, 0)
        st = self.lib.oracle_streamk_embed(_ptr(cover), _ptr(out), cover.size, int(k),
                                           int(geom is not None), W, H, C, p, _ptr(msg),
                                           msg.size, int(bool(header)))
        return st, out

    def streamk_extract(self, stego, k, cap=None, header=True, raw_len=0, geom=None):
        stego = np.ascontiguousarray(stego, dtype=np.uint8).reshape(-1)
        if cap is None:
            cap = stego.size // 2 + 1
        msg = np.full(max(int(cap), 1), STALE, dtype=np.uint8)
        n = _u64(0)
        W, H, C, p = geom if geom is not None else (0, 0, 0, 0)
        st = self.lib.oracle_streamk_extract(_ptr(stego), stego.size, int(k), int(geom is not None),
                                             W, H, C, p, _ptr(msg), int(cap), int(bool(header)),
                                             int(raw_len), ctypes.byref(n))
        return st, msg[: n.value].copy()

    # -- paper2 ----------------------------------------------------------
    def paper2_capacity(self, W, H):
        return int(self.lib.oracle_paper2_capacity(W, H))

    def paper2_embed(self, cover, W, H, Cch, plane, msg, out=None):
        cover = np.ascontiguousarray(cover, dtype=np.uint8).reshape(-1)
        msg = np.ascontiguousarray(msg, dtype=np.uint8).reshape(-1)
        if out is None:
            out = np.zeros_like(cover)
        st = self.lib.oracle_paper2_embed(_ptr(cover), _ptr(out), W, H, Cch, plane,
                                          _ptr(msg), msg.size)
        return st, out

    def paper2_extract(self, stego, W, H, Cch, plane, N, cap=None):
        stego = np.ascontiguousarray(stego, dtype=np.uint8).reshape(-1)
        if cap is None:
            cap = N
        msg = np.full(max(int(cap), 1), STALE, dtype=np.uint8)
        st = self.lib.oracle_paper2_extract(_ptr(stego), W, H, Cch, plane, _ptr(msg),
                                            int(cap), int(N))
        return st, (msg[:N].copy() if st == OK else np.zeros(0, np.uint8))

    # -- statistics ------------------------------------------------------
    def psnr(self, sse: int, n: int) -> float:
        """The module-level ``psnr``; a method so that the pins can be run
        against a handle whose PSNR formula has been replaced."""
        return psnr(sse, n)

    def changed_bytes(self, a, b):
        a = np.ascontiguousarray(a, dtype=np.uint8).reshape(-1)
        b = np.ascontiguousarray(b, dtype=np.uint8).reshape(-1)
        assert a.size == b.size
        c, s = _u64(0), _u64(0)
        self.lib.oracle_changed_bytes(_ptr(a), _ptr(b), a.size, ctypes.byref(c),
                                      ctypes.byref(s))
        return int(c.value), int(s.value)


def psnr(sse: int, n: int) -> float:
    """Section VIII quality measure: PSNR = 10 log10(peak^2 / MSE) with peak
    255 (uint8) and MSE = sse / n, the squared error averaged over all n
    cover bytes (every channel); infinite for an unchanged cover."""
    if sse == 0:
        return math.inf
    return 10.0 * math.log10(255.0 * 255.0 * n / sse)


_DEFAULT = None


def load(rebuild: bool = False) -> Oracle:
    """Build (if needed) and load the default oracle library."""
    global _DEFAULT
    if _DEFAULT is None or rebuild:
        if rebuild or not os.path.exists(_LIB) or \
                os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            build()
        _DEFAULT = Oracle(_LIB)
    return _DEFAULT
