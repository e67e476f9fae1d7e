"""Helpers for the GPU parity tests: guarded device buffers (canary bytes on
both sides, chosen misalignment) and host/device transfers."""
from __future__ import annotations

import os

import numpy as np
import pytest
import torch

GUARD = 256          # canary bytes on each side of an output buffer
CANARY = 0xA7


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0912_0947_gb300 import build
    build.build()
    import paper_0912_0947_gb300 as S
    return S


class Guarded:
    """A device buffer of n bytes starting `off` bytes past a 256-byte
    aligned address, surrounded by canary bytes."""

    def __init__(self, n: int, off: int = 0, fill: np.ndarray | int | None = None,
                 device="cuda"):
        self.n, self.off = n, off
        self.full = torch.full((GUARD + off + n + GUARD,), CANARY, dtype=torch.uint8,
                               device=device)
        self.view = self.full[GUARD + off: GUARD + off + n]
        if fill is not None:
            if isinstance(fill, int):
                self.view.fill_(fill)
            else:
                self.view.copy_(torch.from_numpy(np.ascontiguousarray(fill)).to(device))

    def host(self) -> np.ndarray:
        return self.view.cpu().numpy()

    def canaries_intact(self) -> bool:
        f = self.full.cpu().numpy()
        head = f[: GUARD + self.off]
        tail = f[GUARD + self.off + self.n:]
        return bool(np.all(head == CANARY) and np.all(tail == CANARY))


def dev(a: np.ndarray, device="cuda") -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a)).to(device)


def host_threads() -> int:
    """Host cores this process may run on."""
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return max(1, os.cpu_count() or 1)


def pmap(fn, n: int, workers: int | None = None) -> list:
    """[fn(i) for i in range(n)] on a thread pool over every host core.  The
    oracle's work is one C call per item, which runs without the interpreter
    lock, so the items proceed in parallel."""
    import concurrent.futures as cf
    with cf.ThreadPoolExecutor(max_workers=workers or host_threads()) as ex:
        return list(ex.map(fn, range(n)))
