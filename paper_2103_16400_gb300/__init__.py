"""hexgpu: negacyclic NTT and element-wise modular kernels for one GB300.

The compute lives in the C-ABI library ``libhexgpu.so`` (hand-written
sm_103a CUDA, declared in ``include/hexgpu.h``); ``capi`` is its ctypes
binding with the same function names, and ``tensors`` holds the small torch
helpers (uint64 storage in int64 tensors, host/device copies) that the
tests, the benchmark and the serving loop share.  torch provides device
memory and streams only.
"""
from .capi import HexError, Plan, load  # noqa: F401
from . import capi  # noqa: F401

__all__ = ["HexError", "Plan", "load", "capi"]
