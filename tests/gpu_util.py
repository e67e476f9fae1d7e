"""Helpers for the GPU parity tests: guarded device buffers (canary bytes on
both sides, chosen misalignment) and host/device transfers."""
from __future__ import annotations

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
