"""uint64 coefficient buffers held in torch int64 tensors (same bits).

torch supplies device memory, pinned host memory and streams; the bits are
reinterpreted, never converted, so values up to 2^64 - 1 round-trip exactly.
"""
from __future__ import annotations

import numpy as np
import torch


def to_device(x: np.ndarray, device="cuda") -> torch.Tensor:
    a = np.ascontiguousarray(x, dtype=np.uint64).view(np.int64)
    return torch.from_numpy(a.copy()).to(device)


def to_host(t: torch.Tensor) -> np.ndarray:
    return t.detach().to("cpu").contiguous().numpy().view(np.uint64)


def empty(shape, device="cuda") -> torch.Tensor:
    return torch.empty(tuple(shape), dtype=torch.int64, device=device)


def pinned_from(x: np.ndarray) -> torch.Tensor:
    a = np.ascontiguousarray(x, dtype=np.uint64).view(np.int64)
    return torch.from_numpy(a.copy()).pin_memory()
