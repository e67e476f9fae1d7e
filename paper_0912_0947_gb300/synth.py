"""Seeded synthetic inputs (covers, messages, video frames, uneven batches,
arrival streams).

This module holds no steganography arithmetic: it only draws bytes.  Tests
feed the same arrays to the CPU oracle and to the CUDA path, and the bench
uses it to build its workloads.

Random numbers come from splitmix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: 64-bit word k of stream ``seed`` is ``mix(seed + (k+1)*GAMMA)``
with the published finaliser constants.  Byte i of a byte stream is byte
``i % 8`` (little-endian) of word ``i // 8``.  The same words can therefore be
produced in any chunking, on the host (numpy, pure Python) or on a CUDA device
(torch integer ops), and they agree bit for bit.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

GAMMA = 0x9E3779B97F4A7C15
M1 = 0xBF58476D1CE4E5B9
M2 = 0x94D049BB133111EB
MASK64 = (1 << 64) - 1

# base seed of each workload: 0xC0FFEE00 + workload number
SEED_BASE = 0xC0FFEE00


def _signed(v: int) -> int:
    v &= MASK64
    return v - (1 << 64) if v >= (1 << 63) else v


def splitmix64_py(seed: int, k: int) -> int:
    """Word k of stream ``seed`` (pure Python; the definition)."""
    z = (seed + (k + 1) * GAMMA) & MASK64
    z = ((z ^ (z >> 30)) * M1) & MASK64
    z = ((z ^ (z >> 27)) * M2) & MASK64
    return z ^ (z >> 31)


def substream(seed: int, tag: int) -> int:
    """Seed of an independent stream derived from ``seed`` by ``tag``."""
    return splitmix64_py(seed ^ 0x5DEECE66D, tag)


def words_np(seed: int, k0: int, n: int) -> np.ndarray:
    """Words k0..k0+n-1 of stream ``seed`` as uint64 (numpy, wrapping)."""
    with np.errstate(over="ignore"):
        k = np.arange(k0 + 1, k0 + n + 1, dtype=np.uint64)
        z = np.uint64(seed & MASK64) + k * np.uint64(GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(M1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(M2)
        return z ^ (z >> np.uint64(31))


def _srl(z: torch.Tensor, s: int) -> torch.Tensor:
    """Logical right shift of an int64 tensor viewed as uint64."""
    return (z >> s) & ((1 << (64 - s)) - 1)


def words_torch(seed: int, k0: int, n: int, device="cpu") -> torch.Tensor:
    """Words k0..k0+n-1 of stream ``seed`` as int64 (two's complement of the
    uint64 value), computed with torch integer ops on ``device``."""
    k = torch.arange(k0 + 1, k0 + n + 1, dtype=torch.int64, device=device)
    z = k * _signed(GAMMA) + _signed(seed)
    z = (z ^ _srl(z, 30)) * _signed(M1)
    z = (z ^ _srl(z, 27)) * _signed(M2)
    return z ^ _srl(z, 31)


_CHUNK_WORDS = 1 << 24  # 128 MiB of output per chunk keeps temporaries small


def uniform_bytes(n: int, seed: int, device="cpu", out: torch.Tensor | None = None) -> torch.Tensor:
    """n bytes of stream ``seed`` as a uint8 tensor on ``device``."""
    n = int(n)
    if out is None:
        out = torch.empty(n, dtype=torch.uint8, device=device)
    nw = (n + 7) // 8
    for w0 in range(0, nw, _CHUNK_WORDS):
        cnt = min(_CHUNK_WORDS, nw - w0)
        b = words_torch(seed, w0, cnt, device=out.device).view(torch.uint8)
        lo = w0 * 8
        hi = min(n, lo + cnt * 8)
        out[lo:hi] = b[: hi - lo]
    return out


def uniform_bytes_np(n: int, seed: int) -> np.ndarray:
    """Host copy of ``uniform_bytes`` (numpy)."""
    nw = (int(n) + 7) // 8
    return words_np(seed, 0, nw).view(np.uint8)[: int(n)].copy()


def uniform_floats_np(n: int, seed: int) -> np.ndarray:
    """n doubles in [0, 1): the top 53 bits of each word times 2**-53."""
    w = words_np(seed, 0, int(n))
    return (w >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


# --------------------------------------------------------------------------
# Workloads
# --------------------------------------------------------------------------

STREAM_HEADER_BYTES = 4  # 32-bit bit-count header in front of the message


def stream1_capacity(cover_bytes: int, header: bool = True) -> int:
    """Message bytes that fit one bit per cover byte (header included)."""
    cap = cover_bytes // 8 - (STREAM_HEADER_BYTES if header else 0)
    return max(cap, 0)


@dataclass
class Single:
    """One interleaved uint8 cover and a message."""
    name: str
    height: int
    width: int
    channels: int
    msg_bytes: int
    seed: int

    @property
    def cover_bytes(self) -> int:
        return self.height * self.width * self.channels

    def cover(self, device="cpu") -> torch.Tensor:
        return uniform_bytes(self.cover_bytes, substream(self.seed, 1), device)

    def message(self, device="cpu") -> torch.Tensor:
        return uniform_bytes(self.msg_bytes, substream(self.seed, 2), device)


def single_512() -> Single:
    """512x512x3 uniform cover, 32768-byte uniform message (~1/3 capacity)."""
    return Single("single 512x512x3, 32768 B message", 512, 512, 3, 32768, SEED_BASE + 1)


def single_8192() -> Single:
    """8192x8192x3 uniform cover (201 MB) with a message at full 1-bit
    capacity: 201326592/8 - 4 = 25165820 bytes."""
    C = 8192 * 8192 * 3
    return Single("single 8192x8192x3, full capacity", 8192, 8192, 3,
                  stream1_capacity(C), SEED_BASE + 2)


@dataclass
class Video:
    """F frames of H x W x 3: a smooth gradient plus uniform noise in [0, 16),
    and one message stream split across frames, P bytes per frame, each frame
    with its own header, header+payload = half the frame's 1-bit capacity."""
    frames: int = 600
    height: int = 1080
    width: int = 1920
    channels: int = 3
    seed: int = SEED_BASE + 3

    @property
    def frame_bytes(self) -> int:
        return self.height * self.width * self.channels

    @property
    def per_frame_msg(self) -> int:
        return self.frame_bytes // 2 // 8 - STREAM_HEADER_BYTES

    def frame_range(self, f0: int, f1: int, device="cpu") -> torch.Tensor:
        """Frames [f0, f1) as a (f1-f0, H, W, C) uint8 tensor.
        g(f,y,x,c) = ((x*239)//(W-1) + (y*239)//(H-1))//2 + 7c + f, mod 240,
        plus noise byte & 15 (maximum 254, no clamp needed)."""
        H, W, Cc = self.height, self.width, self.channels
        n = f1 - f0
        y = torch.arange(H, device=device, dtype=torch.int32).view(1, H, 1, 1)
        x = torch.arange(W, device=device, dtype=torch.int32).view(1, 1, W, 1)
        c = torch.arange(Cc, device=device, dtype=torch.int32).view(1, 1, 1, Cc)
        f = torch.arange(f0, f1, device=device, dtype=torch.int32).view(n, 1, 1, 1)
        g = (((x * 239) // (W - 1) + (y * 239) // (H - 1)) // 2 + 7 * c + f) % 240
        out = torch.empty((n, H, W, Cc), dtype=torch.uint8, device=device)
        fb = self.frame_bytes
        for i in range(n):
            noise = uniform_bytes(fb, substream(self.seed, 1000 + f0 + i), device)
            out[i] = (g[i] + (noise.view(H, W, Cc).to(torch.int32) & 15)).to(torch.uint8)
        return out

    def message(self, device="cpu") -> torch.Tensor:
        """The whole stream, frames * per_frame_msg bytes."""
        return uniform_bytes(self.frames * self.per_frame_msg, substream(self.seed, 2), device)


@dataclass
class UnevenItem:
    width: int
    height: int
    channels: int
    msg_bytes: int
    seed: int

    @property
    def cover_bytes(self) -> int:
        return self.width * self.height * self.channels


def uneven_batch(count: int = 4096, seed: int = SEED_BASE + 4, lo: int = 64, hi: int = 4096,
                 fill_lo: float = 0.05, fill_hi: float = 1.0) -> list[UnevenItem]:
    """Covers whose width and height are independently log-uniform in
    [lo, hi] (rounded), half grayscale (1 channel) and half RGB (3), each
    with a message of floor(f * capacity) bytes, f uniform in
    [fill_lo, fill_hi], capacity = the 1-bit capacity with header."""
    u = uniform_floats_np(4 * count, substream(seed, 7)).reshape(count, 4)
    la, lb = math.log(lo), math.log(hi)
    items = []
    for i in range(count):
        w = int(round(math.exp(la + (lb - la) * u[i, 0])))
        h = int(round(math.exp(la + (lb - la) * u[i, 1])))
        ch = 1 if u[i, 2] < 0.5 else 3
        cap = stream1_capacity(w * h * ch)
        f = fill_lo + (fill_hi - fill_lo) * u[i, 3]
        items.append(UnevenItem(w, h, ch, int(math.floor(f * cap)), substream(seed, 100 + i)))
    return items


def poisson_arrivals(rate_hz: float, count: int, seed: int) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process: exponential gaps
    -ln(1-U)/rate, cumulatively summed."""
    u = uniform_floats_np(count, seed)
    return np.cumsum(-np.log1p(-u) / rate_hz)
