"""Helpers for the GPU parity tests: guarded device buffers at chosen byte offsets.

Every output buffer is surrounded by guard bytes filled with a known pattern;
after each call the guards are checked, which catches out-of-bounds writes
(compute-sanitizer is not used on the test machines).
"""
from __future__ import annotations

import numpy as np
import torch

GUARD = 64
PATTERN = 0xA5


class Guarded:
    """A device byte buffer with `nbytes` usable bytes starting at byte offset `off`."""

    def __init__(self, nbytes: int, off: int = 0, fill: np.ndarray | None = None,
                 fill_byte: int = PATTERN):
        self.nbytes = nbytes
        self.off = off
        total = GUARD + 16 + nbytes + GUARD
        self.start = GUARD + off        # GUARD is a multiple of 16, so alignment == off % 16
        self.buf = torch.full((total,), fill_byte, dtype=torch.uint8, device="cuda")
        if fill is not None:
            raw = np.ascontiguousarray(fill).view(np.uint8).reshape(-1)
            assert raw.size == nbytes
            self.buf[self.start:self.start + nbytes] = torch.from_numpy(raw.copy()).cuda()

    @property
    def ptr(self) -> int:
        return self.buf.data_ptr() + self.start

    def inner(self) -> np.ndarray:
        return self.buf[self.start:self.start + self.nbytes].cpu().numpy()

    def check_guards(self, fill_byte: int = PATTERN) -> None:
        h = self.buf.cpu().numpy()
        before = h[:self.start]
        after = h[self.start + self.nbytes:]
        assert np.all(before == fill_byte), "write before the output buffer"
        assert np.all(after == fill_byte), "write after the output buffer"


def span_bytes(n: int, inc: int, elem: int) -> int:
    """Bytes covered by n elements of `elem` bytes at element stride inc."""
    return 0 if n == 0 else ((n - 1) * inc + 1) * elem


def sync():
    torch.cuda.synchronize()
