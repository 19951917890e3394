"""The C-ABI library builds, loads without a GPU, exports every function that
include/hexgpu.h declares, and rejects bad arguments on the host before any
CUDA call (no compute here: these run on CPU)."""
import ctypes
import os
import re

import pytest

import workloads as W
from paper_2103_16400_gb300 import build, capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return capi.load()


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(hx_[a-z0-9_]+)\s*\(",
                            text, flags=re.M)
    return names


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("hx_plan_create", "hx_ntt_forward", "hx_ntt_inverse", "hx_ntt_forward_raw",
                 "hx_eltwise_add_mod", "hx_eltwise_mult_mod", "hx_eltwise_fma_mod",
                 "hx_poly_mul", "hx_ciphertext_tensor", "hx_strerror"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    # and the binding wraps each one under the same name
    assert set(declared_functions()) <= set(capi.exported_symbols())


def test_strerror_and_version(lib):
    assert lib.hx_abi_version() == 1
    assert lib.hx_strerror(0) == b"success"
    assert b"power of two" in lib.hx_strerror(-3)


def _plan_status(lib, N, moduli, roots=None):
    h = ctypes.c_void_p()
    return lib.hx_plan_create(ctypes.byref(h), N, capi.host_u64(moduli), len(moduli),
                              capi.host_u64(roots) if roots else None)


def test_plan_validation_on_host(lib):
    q = W.ntt_primes(50, 2048, 1)[0]
    assert _plan_status(lib, 1000, [q]) == -3            # not a power of two
    assert _plan_status(lib, 512, [q]) == -3             # below 2^10
    assert _plan_status(lib, 1 << 18, [q]) == -3         # above 2^17
    assert _plan_status(lib, 4096, [q]) == -4            # q != 1 mod 2N
    assert _plan_status(lib, 1024, [q + 2048]) == -4     # not prime
    big = W.ntt_primes(63, 2048, 1)[0]
    assert _plan_status(lib, 1024, [big]) == -4          # q >= 2^62
    assert _plan_status(lib, 1024, [q], roots=[5]) == -5  # not a primitive root
    assert lib.hx_plan_create(None, 1024, capi.host_u64([q]), 1, None) == -1
    assert _plan_status(lib, 1024, []) in (-8, -1)


def test_elementwise_validation_on_host(lib):
    m = capi.host_u64([97])
    assert lib.hx_eltwise_add_mod(None, 16, 16, 8, m, 1, 1, None) == -1
    assert lib.hx_eltwise_add_mod(16, 16, 16, 0, m, 1, 1, None) == -8
    assert lib.hx_eltwise_add_mod(24, 16, 16, 8, m, 1, 1, None) == -2
    assert lib.hx_eltwise_add_mod(32, 16, 16, 8, m, 1, 1, None) == -9   # partial overlap
    assert lib.hx_eltwise_mult_mod(16, 16, 16, 8, m, 1, 1, 3, None) == -6
    assert lib.hx_eltwise_mult_mod(16, 16, 16, 8, capi.host_u64([1 << 40]), 1, 1, 1, None) == -4
    assert lib.hx_eltwise_fma_mod(16, 16, capi.host_u64([1]), None, 8,
                                  capi.host_u64([1 << 62]), 1, 1, 1, None) == -4
    assert lib.hx_ntt_forward(None, 16, 16, 1, 1, 1, None) == -1
