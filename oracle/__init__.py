"""CPU oracle for the negacyclic NTT, the cyclic NTT and the element-wise
modular kernels.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The CUDA library never
imports, links or runs anything here, and nothing here imports the CUDA
library.  Both sides receive inputs from the separate ``workloads`` module.

Two layers:
  * ``hx_oracle.c``: plain C with the naive 128-bit ``%`` modular product of
    Listing 1 (Section 2.1); radix-2 Cooley-Tukey forward and Gentleman-Sande
    inverse exactly as the paper's two NTT algorithms state them (Section 2.2);
    closed-form and schoolbook evaluators; element-wise definitions
    (addition, subtraction, negation, products, FMA); the cyclic NTT, its
    inverse and the cyclic product written out from their Section 2.2
    definitions.
  * ``oracle.bigint``: pure-Python big-integer definitions for tiny N, written
    from the definitions alone (no transform algorithm), used to pin the C code.

The composite functions below (polynomial product, ciphertext tensor) are
compositions of those calls in the order the paper's Listing 4 gives.

Parity status: every function here is pinned by the ``-m "not gpu"`` tests
(closed forms, brute force, invariants, library routines); none is unpinned.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hx_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libhx_oracle.so")
_lock = threading.Lock()
_lib = None

U64 = ctypes.c_uint64
P64 = ctypes.POINTER(ctypes.c_uint64)


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc into oracle/_build (no CUDA involved)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or \
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            for name in ("oracle_mulmod", "oracle_addmod", "oracle_submod",
                         "oracle_powmod"):
                getattr(L, name).restype = U64
                getattr(L, name).argtypes = [U64, U64, U64]
            L.oracle_invmod.restype = U64
            L.oracle_invmod.argtypes = [U64, U64]
            L.oracle_is_prime.restype = ctypes.c_int
            L.oracle_is_prime.argtypes = [U64]
            L.oracle_min_primitive_root.restype = U64
            L.oracle_min_primitive_root.argtypes = [U64, U64]
            L.oracle_bitrev_powers.restype = None
            L.oracle_bitrev_powers.argtypes = [U64, U64, U64, P64]
            for name in ("oracle_ntt_forward", "oracle_ntt_inverse"):
                getattr(L, name).restype = None
                getattr(L, name).argtypes = [P64, U64, U64, P64]
            L.oracle_ntt_forward_direct.restype = None
            L.oracle_ntt_forward_direct.argtypes = [P64, U64, U64, U64, P64, U64, P64]
            L.oracle_negacyclic_schoolbook.restype = None
            L.oracle_negacyclic_schoolbook.argtypes = [P64, P64, U64, U64, P64, U64, P64]
            for name in ("oracle_eltwise_add_mod", "oracle_eltwise_sub_mod",
                         "oracle_eltwise_mult_mod"):
                getattr(L, name).restype = None
                getattr(L, name).argtypes = [P64, P64, P64, U64, U64]
            L.oracle_eltwise_fma_mod.restype = None
            L.oracle_eltwise_fma_mod.argtypes = [P64, P64, U64, P64, U64, U64]
            L.oracle_eltwise_negate_mod.restype = None
            L.oracle_eltwise_negate_mod.argtypes = [P64, P64, U64, U64]
            L.oracle_min_primitive_nth_root.restype = U64
            L.oracle_min_primitive_nth_root.argtypes = [U64, U64]
            L.oracle_cyclic_ntt_direct.restype = None
            L.oracle_cyclic_ntt_direct.argtypes = [P64, U64, U64, U64, P64, U64, P64]
            L.oracle_cyclic_intt_direct.restype = None
            L.oracle_cyclic_intt_direct.argtypes = [P64, U64, U64, U64, P64]
            L.oracle_cyclic_schoolbook.restype = None
            L.oracle_cyclic_schoolbook.argtypes = [P64, P64, U64, U64, P64, U64, P64]
            _lib = L
    return _lib


def _p(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.dtype == np.uint64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(P64)


# ---------------------------------------------------------------- scalars
def mulmod(a: int, b: int, q: int) -> int:
    return int(lib().oracle_mulmod(a, b, q))


def powmod(a: int, e: int, q: int) -> int:
    return int(lib().oracle_powmod(a, e, q))


def invmod(a: int, q: int) -> int:
    return int(lib().oracle_invmod(a, q))


def is_prime(n: int) -> bool:
    return bool(lib().oracle_is_prime(n))


def min_primitive_root(N: int, q: int) -> int:
    """Smallest primitive 2N-th root of unity mod q (0 if none / bad input)."""
    return int(lib().oracle_min_primitive_root(N, q))


def min_primitive_nth_root(N: int, q: int) -> int:
    """Smallest primitive N-th root of unity mod q (0 if none / bad input)."""
    return int(lib().oracle_min_primitive_nth_root(N, q))


def bitrev_powers(N: int, q: int, root: int) -> np.ndarray:
    t = np.empty(N, dtype=np.uint64)
    lib().oracle_bitrev_powers(N, q, root, _p(t))
    return t


class Tables:
    """Per-(N, q) oracle tables: psi, psi_rev, psi^-1_rev (Section 2.2)."""

    def __init__(self, N: int, q: int, psi: Optional[int] = None):
        self.N, self.q = N, q
        self.psi = psi if psi is not None else min_primitive_root(N, q)
        if self.psi == 0:
            raise ValueError(f"no primitive 2N-th root for N={N}, q={q}")
        self.psi_inv = invmod(self.psi, q)
        self.psi_rev = bitrev_powers(N, q, self.psi)
        self.psiinv_rev = bitrev_powers(N, q, self.psi_inv)


_tables_cache = {}


def tables(N: int, q: int, psi: Optional[int] = None) -> Tables:
    key = (N, q, psi)
    if key not in _tables_cache:
        _tables_cache[key] = Tables(N, q, psi)
    return _tables_cache[key]


# ---------------------------------------------------------------- one limb
def ntt_forward_1(x: np.ndarray, q: int, psi: Optional[int] = None,
                  psi_rev: Optional[np.ndarray] = None) -> np.ndarray:
    """Forward negacyclic NTT of one length-N vector (bit-reversed output)."""
    a = np.ascontiguousarray(x, dtype=np.uint64).copy()
    N = len(a)
    if psi_rev is None:
        psi_rev = tables(N, q, psi).psi_rev
    lib().oracle_ntt_forward(_p(a), N, q, _p(np.ascontiguousarray(psi_rev)))
    return a


def ntt_inverse_1(x: np.ndarray, q: int, psi: Optional[int] = None,
                  psiinv_rev: Optional[np.ndarray] = None) -> np.ndarray:
    """Inverse negacyclic NTT of one vector (bit-reversed input)."""
    a = np.ascontiguousarray(x, dtype=np.uint64).copy()
    N = len(a)
    if psiinv_rev is None:
        psiinv_rev = tables(N, q, psi).psiinv_rev
    lib().oracle_ntt_inverse(_p(a), N, q, _p(np.ascontiguousarray(psiinv_rev)))
    return a


def ntt_forward_direct(x: np.ndarray, q: int, psi: int, idx: Sequence[int]) -> np.ndarray:
    """Closed-form forward NTT outputs at the given indices, O(N) each."""
    a = np.ascontiguousarray(x, dtype=np.uint64)
    ix = np.ascontiguousarray(np.asarray(idx, dtype=np.uint64))
    out = np.empty(len(ix), dtype=np.uint64)
    lib().oracle_ntt_forward_direct(_p(a), len(a), q, psi, _p(ix), len(ix), _p(out))
    return out


def negacyclic_schoolbook(a: np.ndarray, b: np.ndarray, q: int,
                          idx: Optional[Sequence[int]] = None) -> np.ndarray:
    """O(N) per output negacyclic product coefficients (all if idx is None)."""
    a = np.ascontiguousarray(a, dtype=np.uint64)
    b = np.ascontiguousarray(b, dtype=np.uint64)
    N = len(a)
    if idx is None:
        out = np.empty(N, dtype=np.uint64)
        lib().oracle_negacyclic_schoolbook(_p(a), _p(b), N, q, None, 0, _p(out))
    else:
        ix = np.ascontiguousarray(np.asarray(idx, dtype=np.uint64))
        out = np.empty(len(ix), dtype=np.uint64)
        lib().oracle_negacyclic_schoolbook(_p(a), _p(b), N, q, _p(ix), len(ix), _p(out))
    return out


def _elt2(fn, a, b, q):
    a = np.ascontiguousarray(a, dtype=np.uint64)
    b = np.ascontiguousarray(b, dtype=np.uint64)
    c = np.empty_like(a)
    getattr(lib(), fn)(_p(c), _p(a), _p(b), len(a), q)
    return c


def eltwise_add_mod_1(a, b, q):
    return _elt2("oracle_eltwise_add_mod", a, b, q)


def eltwise_sub_mod_1(a, b, q):
    return _elt2("oracle_eltwise_sub_mod", a, b, q)


def eltwise_mult_mod_1(a, b, q):
    return _elt2("oracle_eltwise_mult_mod", a, b, q)


def eltwise_fma_mod_1(a, s: int, d, q):
    a = np.ascontiguousarray(a, dtype=np.uint64)
    dd = None if d is None else np.ascontiguousarray(d, dtype=np.uint64)
    c = np.empty_like(a)
    lib().oracle_eltwise_fma_mod(_p(c), _p(a), int(s), _p(dd), len(a), q)
    return c


def eltwise_negate_mod_1(a, q):
    a = np.ascontiguousarray(a, dtype=np.uint64)
    c = np.empty_like(a)
    lib().oracle_eltwise_negate_mod(_p(c), _p(a), len(a), q)
    return c


def cyclic_ntt_1(x: np.ndarray, q: int, omega: int, idx: Optional[Sequence[int]] = None):
    """Cyclic NTT by definition (Section 2.2), natural order: outputs i in idx
    (all N when idx is None), O(N) each."""
    a = np.ascontiguousarray(x, dtype=np.uint64)
    N = len(a)
    ix = np.arange(N, dtype=np.uint64) if idx is None else \
        np.ascontiguousarray(np.asarray(idx, dtype=np.uint64))
    out = np.empty(len(ix), dtype=np.uint64)
    lib().oracle_cyclic_ntt_direct(_p(a), N, q, omega, _p(ix), len(ix), _p(out))
    return out


def cyclic_intt_1(x: np.ndarray, q: int, omega: int) -> np.ndarray:
    """Inverse cyclic NTT by definition (Section 2.2), natural order, O(N^2)."""
    a = np.ascontiguousarray(x, dtype=np.uint64)
    out = np.empty_like(a)
    lib().oracle_cyclic_intt_direct(_p(a), len(a), q, omega, _p(out))
    return out


def cyclic_schoolbook(a: np.ndarray, b: np.ndarray, q: int,
                      idx: Optional[Sequence[int]] = None) -> np.ndarray:
    """Product in Z_q[X] / (X^N - 1), O(N) per output (all if idx is None)."""
    a = np.ascontiguousarray(a, dtype=np.uint64)
    b = np.ascontiguousarray(b, dtype=np.uint64)
    N = len(a)
    if idx is None:
        out = np.empty(N, dtype=np.uint64)
        lib().oracle_cyclic_schoolbook(_p(a), _p(b), N, q, None, 0, _p(out))
    else:
        ix = np.ascontiguousarray(np.asarray(idx, dtype=np.uint64))
        out = np.empty(len(ix), dtype=np.uint64)
        lib().oracle_cyclic_schoolbook(_p(a), _p(b), N, q, _p(ix), len(ix), _p(out))
    return out


# ---------------------------------------------------------------- batches
# Arrays are [n_polys, n_limbs, N]; limb l is reduced modulo moduli[l].
def ntt_forward(x: np.ndarray, moduli: Sequence[int], psis: Optional[Sequence[int]] = None):
    out = np.empty_like(x)
    for p in range(x.shape[0]):
        for l, q in enumerate(moduli):
            out[p, l] = ntt_forward_1(x[p, l], int(q), None if psis is None else psis[l])
    return out


def ntt_inverse(x: np.ndarray, moduli: Sequence[int], psis: Optional[Sequence[int]] = None):
    out = np.empty_like(x)
    for p in range(x.shape[0]):
        for l, q in enumerate(moduli):
            out[p, l] = ntt_inverse_1(x[p, l], int(q), None if psis is None else psis[l])
    return out


def eltwise_add_mod(a, b, moduli):
    out = np.empty_like(a)
    for p in range(a.shape[0]):
        for l, q in enumerate(moduli):
            out[p, l] = eltwise_add_mod_1(a[p, l], b[p, l], int(q))
    return out


def eltwise_negate_mod(a, moduli):
    out = np.empty_like(a)
    for p in range(a.shape[0]):
        for l, q in enumerate(moduli):
            out[p, l] = eltwise_negate_mod_1(a[p, l], int(q))
    return out


def eltwise_mult_mod(a, b, moduli):
    out = np.empty_like(a)
    for p in range(a.shape[0]):
        for l, q in enumerate(moduli):
            out[p, l] = eltwise_mult_mod_1(a[p, l], b[p, l], int(q))
    return out


def eltwise_fma_mod(a, s, d, moduli):
    out = np.empty_like(a)
    for p in range(a.shape[0]):
        for l, q in enumerate(moduli):
            out[p, l] = eltwise_fma_mod_1(a[p, l], int(s[l]),
                                          None if d is None else d[p, l], int(q))
    return out


def poly_mul(a: np.ndarray, b: np.ndarray, moduli: Sequence[int]) -> np.ndarray:
    """Negacyclic product in R_q per limb, composed as in Listing 4:
    forward NTT of both operands, element-wise product, inverse NTT."""
    fa = ntt_forward(a, moduli)
    fb = ntt_forward(b, moduli)
    return ntt_inverse(eltwise_mult_mod(fa, fb, moduli), moduli)


def ciphertext_tensor(a0, a1, b0, b1, s, e0, e1, e2, moduli):
    """Tensor product of two degree-1 ciphertexts followed by a scaled
    accumulation, composed from the element-wise definitions:
      (A0, A1, B0, B1) = forward NTT of (a0, a1, b0, b1)
      d0 = A0*B0,  d1 = A0*B1 + A1*B0,  d2 = A1*B1        (Section 2 products)
      r_k = d_k * s_l + e_k                                  (EltwiseFMAMod)
      out_k = inverse NTT of r_k.
    Arrays are [n_polys, n_limbs, N]; s has one scalar per limb."""
    A0, A1, B0, B1 = (ntt_forward(x, moduli) for x in (a0, a1, b0, b1))
    d0 = eltwise_mult_mod(A0, B0, moduli)
    d1 = eltwise_add_mod(eltwise_mult_mod(A0, B1, moduli),
                         eltwise_mult_mod(A1, B0, moduli), moduli)
    d2 = eltwise_mult_mod(A1, B1, moduli)
    rs = [eltwise_fma_mod(d, s, e, moduli) for d, e in ((d0, e0), (d1, e1), (d2, e2))]
    return tuple(ntt_inverse(r, moduli) for r in rs)
