"""Thin ctypes binding to libhexgpu.so, with the C ABI's own names.

Argument marshalling only: device buffers are passed as raw pointers (a torch
CUDA tensor's data_ptr(), or an int), host arrays are copied into ctypes
arrays, streams default to torch's current stream.  Every computation runs
in the CUDA library; there is no CPU path.  A non-zero status raises
HexError carrying the library's own message.
"""
from __future__ import annotations

import ctypes
import functools
import os
import threading
from typing import Optional, Sequence

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhexgpu.so")

U32, U64, I32 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
VP = ctypes.c_void_p
P64 = ctypes.POINTER(ctypes.c_uint64)

# name -> argtypes (restype int unless listed in _RESTYPES)
_SIGS = {
    "hx_strerror": [I32],
    "hx_abi_version": [],
    "hx_plan_create": [ctypes.POINTER(VP), U64, P64, U32, P64],
    "hx_plan_create_cyclic": [ctypes.POINTER(VP), U64, P64, U32, P64],
    "hx_plan_destroy": [VP],
    "hx_plan_roots": [VP, P64],
    "hx_plan_info": [VP, P64, ctypes.POINTER(U32), P64],
    "hx_plan_set_schedule": [VP, U32, U32, ctypes.POINTER(ctypes.c_int32)],
    "hx_plan_get_schedule": [VP, U32, ctypes.POINTER(U32), ctypes.POINTER(ctypes.c_int32)],
    "hx_ntt_forward": [VP, VP, VP, U32, U32, U32, VP],
    "hx_ntt_inverse": [VP, VP, VP, U32, U32, U32, VP],
    "hx_ntt_forward_raw": [VP, U64, P64, U32, U32, U32, VP],
    "hx_ntt_inverse_raw": [VP, U64, P64, U32, U32, U32, VP],
    "hx_eltwise_add_mod": [VP, VP, VP, U64, P64, U32, U32, VP],
    "hx_eltwise_sub_mod": [VP, VP, VP, U64, P64, U32, U32, VP],
    "hx_eltwise_negate_mod": [VP, VP, U64, P64, U32, U32, VP],
    "hx_eltwise_mult_mod": [VP, VP, VP, U64, P64, U32, U32, U32, VP],
    "hx_eltwise_fma_mod": [VP, VP, P64, VP, U64, P64, U32, U32, U32, VP],
    "hx_poly_mul": [VP, VP, VP, VP, U32, VP],
    "hx_dyadic_inverse": [VP, VP, VP, VP, U32, U32, VP],
    "hx_ciphertext_tensor": [VP, VP, VP, VP, VP, VP, VP, VP, P64, VP, VP, VP, U32, VP],
    "hx_tensor_fma_inverse": [VP, VP, VP, VP, VP, VP, VP, VP, P64, VP, VP, VP, U32, U32, VP],
    "hx_ciphertext_step": [VP, VP, VP, VP, P64, VP, U32, VP],
    "hx_poly_product": [VP, VP, VP, VP, VP, U32, VP],
    "hx_dyadic_tensor_fma": [VP, VP, VP, VP, VP, VP, VP, P64, VP, VP, VP, U64, P64, U32, U32,
                             U32, VP],
    "hx_ragged_set_split": [U32, U32],
    "hx_ragged_get_split": [U32, ctypes.POINTER(U32)],
    "hx_batch_create": [ctypes.POINTER(VP), VP, U32, U32, U32, U32],
    "hx_batch_run": [VP, VP],
    "hx_batch_info": [VP, P64, P64, ctypes.POINTER(U32)],
    "hx_batch_destroy": [VP],
    "hx_batch_run_static": [VP, U32, U32, U32, U32, VP],
    "hx_polymul_ragged_workspace": [VP, U32, P64],
    "hx_polymul_ragged": [VP, U32, VP, U64, VP],
    "hx_launch_count": [],
    "hx_probe_int_mul_rate": [U32, U32, ctypes.POINTER(ctypes.c_double),
                              ctypes.POINTER(ctypes.c_float), VP],
    "hx_probe_butterfly_rate": [U32, U32, U64, ctypes.POINTER(ctypes.c_double),
                                ctypes.POINTER(ctypes.c_float), VP],
    "hx_probe_copy_rate": [VP, VP, U64, U32, U32, ctypes.POINTER(ctypes.c_double),
                           ctypes.POINTER(ctypes.c_float), VP],
    "hx_ntt_ragged_workspace": [VP, U32, P64],
    "hx_ntt_ragged": [VP, U32, U32, U32, U32, VP, U64, VP],
    "hx_timing_enable": [I32, U32],
    "hx_timing_read": [VP, U32, ctypes.POINTER(U32)],
    "hx_kernel_name": [U32, ctypes.c_char_p, U32],
}
_RESTYPES = {"hx_strerror": ctypes.c_char_p, "hx_launch_count": U64}

_lib = None
_lock = threading.Lock()


class HexError(RuntimeError):
    def __init__(self, fn: str, status: int, msg: str):
        super().__init__(f"{fn}: {msg} (status {status})")
        self.status = status


def load():
    """Load the CUDA library; raises if it has not been built (no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(
                    f"libhexgpu.so is not built ({LIB_PATH}); run "
                    "`python -m paper_2103_16400_gb300.build` (needs nvcc)")
            L = ctypes.CDLL(LIB_PATH)
            for name, args in _SIGS.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = _RESTYPES.get(name, I32)
            _lib = L
    return _lib


def exported_symbols() -> Sequence[str]:
    return list(_SIGS)


def _check(fn: str, st: int):
    if st != 0:
        msg = load().hx_strerror(st).decode()
        raise HexError(fn, st, msg)


def ptr(x) -> Optional[int]:
    """Device pointer of a torch tensor (or an int / None)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def host_u64(values) -> ctypes.Array:
    vals = [int(v) for v in values]
    return (ctypes.c_uint64 * len(vals))(*vals)


def _stream(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# --------------------------------------------------------------------- plans
class Plan:
    """Owns an hx_plan_t: device twiddle tables for (N, moduli); negacyclic
    (roots psi of order 2N), or with cyclic=True the cyclic NTT (roots omega
    of order N)."""

    def __init__(self, N: int, moduli: Sequence[int], roots: Optional[Sequence[int]] = None,
                 cyclic: bool = False):
        L = load()
        h = VP()
        mod = host_u64(moduli)
        rts = host_u64(roots) if roots is not None else None
        fn = "hx_plan_create_cyclic" if cyclic else "hx_plan_create"
        _check(fn, getattr(L, fn)(ctypes.byref(h), N, mod, len(moduli), rts))
        self.handle = h.value
        self.cyclic = cyclic
        self.N = N
        self.moduli = [int(q) for q in moduli]
        self.n_limbs = len(moduli)

    def roots(self):
        out = (ctypes.c_uint64 * self.n_limbs)()
        _check("hx_plan_roots", load().hx_plan_roots(self.handle, out))
        return [int(x) for x in out]

    def info(self):
        N, nl, b = U64(), U32(), U64()
        _check("hx_plan_info", load().hx_plan_info(self.handle, ctypes.byref(N),
                                                   ctypes.byref(nl), ctypes.byref(b)))
        return N.value, nl.value, b.value

    FORWARD, INVERSE, BOTH = 1, 2, 3

    def schedule(self, direction: int = 1):
        """Kernel schedule of the forward (1) or inverse (2) transform: a list
        of (s0, K, logGb, logGc, logR, pipe, np) per pass."""
        n, p = U32(), (ctypes.c_int32 * 14)()
        _check("hx_plan_get_schedule",
               load().hx_plan_get_schedule(self.handle, direction, ctypes.byref(n), p))
        return [tuple(p[7 * i:7 * i + 7]) for i in range(n.value)]

    def set_schedule(self, passes, direction: int = 3):
        flat = [int(v) for ps in passes for v in ps]
        arr = (ctypes.c_int32 * len(flat))(*flat)
        _check("hx_plan_set_schedule",
               load().hx_plan_set_schedule(self.handle, direction, len(passes), arr))

    def destroy(self):
        if getattr(self, "handle", None):
            _check("hx_plan_destroy", load().hx_plan_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def _h(plan):
    return plan.handle if isinstance(plan, Plan) else plan


class RaggedItem(ctypes.Structure):
    """hx_ragged_item: polynomials sharing one plan, in a ragged batch."""
    _fields_ = [("plan", VP), ("d_in", VP), ("d_out", VP), ("n_polys", U32),
                ("reserved", U32)]


class PolymulItem(ctypes.Structure):
    """hx_polymul_item: products a * b of polynomials sharing one plan."""
    _fields_ = [("plan", VP), ("d_a", VP), ("d_b", VP), ("d_result", VP), ("n_polys", U32),
                ("reserved", U32)]


def polymul_items(items):
    """ctypes array of PolymulItem from (plan, a, b, result, n_polys) tuples."""
    items = list(items)
    return (PolymulItem * len(items))(*[PolymulItem(_h(p), ptr(a), ptr(b), ptr(r), n, 0)
                                        for p, a, b, r, n in items]), len(items)


def polymul_items_array(plans, a_ptrs, b_ptrs, r_ptrs, n_polys=1):
    """The same hx_polymul_item array built column by column in numpy (for a
    server launching hundreds of items at once): plan handles and device
    pointers as integer sequences or arrays, n_polys a scalar or sequence.
    Returns (array, n), accepted wherever polymul_items()'s pair is."""
    import numpy as np
    n = len(plans)
    arr = np.zeros(n, _polymul_dtype())
    arr["plan"] = plans
    arr["d_a"] = a_ptrs
    arr["d_b"] = b_ptrs
    arr["d_result"] = r_ptrs
    arr["n_polys"] = n_polys
    return arr, n


@functools.lru_cache(maxsize=None)
def _polymul_dtype():
    import numpy as np
    dt = np.dtype([("plan", "<u8"), ("d_a", "<u8"), ("d_b", "<u8"), ("d_result", "<u8"),
                   ("n_polys", "<u4"), ("reserved", "<u4")])
    assert dt.itemsize == ctypes.sizeof(PolymulItem)
    return dt


def _items_ptr(arr):
    """Address of an item array from polymul_items() or polymul_items_array()."""
    if hasattr(arr, "ctypes") and hasattr(arr, "dtype"):     # numpy array
        if not arr.flags["C_CONTIGUOUS"] or arr.dtype != _polymul_dtype():
            raise ValueError("item array must be a contiguous polymul_items_array()")
        return VP(arr.ctypes.data)
    return ctypes.cast(arr, VP)


def hx_polymul_ragged_workspace(items) -> int:
    arr, n = items if isinstance(items, tuple) else polymul_items(items)
    out = U64()
    _check("hx_polymul_ragged_workspace", load().hx_polymul_ragged_workspace(
        _items_ptr(arr), n, ctypes.byref(out)))
    return out.value


def hx_polymul_ragged(items, workspace, workspace_bytes: int, stream=None):
    """items: (plan, a, b, result, n_polys) tuples or a polymul_items() pair."""
    arr, n = items if isinstance(items, tuple) else polymul_items(items)
    _check("hx_polymul_ragged", load().hx_polymul_ragged(
        _items_ptr(arr), n, ptr(workspace), workspace_bytes, _stream(stream)))


def hx_batch_run_static(items, direction: int = 1, input_mod_factor: int = 1,
                        output_mod_factor: int = 1, stream=None):
    """One run of a ragged set of transforms with no device allocation (the
    library's fixed scratch array holds the work list); items as for Batch."""
    items = list(items)
    arr = (RaggedItem * len(items))(*[RaggedItem(_h(p), ptr(i), ptr(o), n, 0)
                                      for p, i, o, n in items])
    _check("hx_batch_run_static", load().hx_batch_run_static(
        ctypes.cast(arr, VP), len(items), direction, input_mod_factor, output_mod_factor,
        _stream(stream)))


def ragged_items_array(plans, in_ptrs, out_ptrs, n_polys=1):
    """hx_ragged_item array built column by column in numpy (plan handles and
    device pointers as integer sequences or arrays).  Returns (array, n)."""
    import numpy as np
    n = len(plans)
    arr = np.zeros(n, _ragged_dtype())
    arr["plan"] = plans
    arr["d_in"] = in_ptrs
    arr["d_out"] = out_ptrs
    arr["n_polys"] = n_polys
    return arr, n


@functools.lru_cache(maxsize=None)
def _ragged_dtype():
    import numpy as np
    dt = np.dtype([("plan", "<u8"), ("d_in", "<u8"), ("d_out", "<u8"), ("n_polys", "<u4"),
                   ("reserved", "<u4")])
    assert dt.itemsize == ctypes.sizeof(RaggedItem)
    return dt


def _ragged_ptr(items):
    """(address, n) of ragged items: (plan, d_in, d_out, n_polys) tuples or a
    ragged_items_array() pair; the returned object keeps the array alive."""
    if isinstance(items, tuple) and len(items) == 2 and hasattr(items[0], "dtype"):
        arr, n = items
        if not arr.flags["C_CONTIGUOUS"] or arr.dtype != _ragged_dtype():
            raise ValueError("item array must be a contiguous ragged_items_array()")
        return VP(arr.ctypes.data), n, arr
    items = list(items)
    arr = (RaggedItem * len(items))(*[RaggedItem(_h(p), ptr(i), ptr(o), n, 0)
                                      for p, i, o, n in items])
    return ctypes.cast(arr, VP), len(items), arr


def hx_ntt_ragged_workspace(items) -> int:
    p, n, _keep = _ragged_ptr(items)
    out = U64()
    _check("hx_ntt_ragged_workspace", load().hx_ntt_ragged_workspace(p, n, ctypes.byref(out)))
    return out.value


def hx_ntt_ragged(items, workspace, workspace_bytes: int, direction: int = 1,
                  input_mod_factor: int = 1, output_mod_factor: int = 1, stream=None):
    """One run of a ragged set of transforms in a caller-owned workspace."""
    p, n, _keep = _ragged_ptr(items)
    _check("hx_ntt_ragged", load().hx_ntt_ragged(p, n, direction, input_mod_factor,
                                                 output_mod_factor, ptr(workspace),
                                                 workspace_bytes, _stream(stream)))


def hx_ragged_set_split(log2_n: int, k1: int):
    """Column-pass stages of ragged transforms at N = 2^log2_n (process-wide)."""
    _check("hx_ragged_set_split", load().hx_ragged_set_split(log2_n, k1))


def hx_ragged_get_split(log2_n: int) -> int:
    k = U32()
    _check("hx_ragged_get_split", load().hx_ragged_get_split(log2_n, ctypes.byref(k)))
    return k.value


class Batch:
    """Owns an hx_batch_t: a ragged set of transforms replayed as one graph.
    items: iterable of (plan, d_in, d_out, n_polys)."""

    def __init__(self, items, direction: int = 1, input_mod_factor: int = 1,
                 output_mod_factor: int = 1):
        items = list(items)
        arr = (RaggedItem * len(items))(*[RaggedItem(_h(p), ptr(i), ptr(o), n, 0)
                                          for p, i, o, n in items])
        self._keep = items                      # plans and buffers outlive the batch
        h = VP()
        _check("hx_batch_create", load().hx_batch_create(
            ctypes.byref(h), ctypes.cast(arr, VP), len(items), direction, input_mod_factor,
            output_mod_factor))
        self.handle = h.value

    def run(self, stream=None):
        _check("hx_batch_run", load().hx_batch_run(self.handle, _stream(stream)))

    def info(self):
        lt, tiles, launches = U64(), U64(), U32()
        _check("hx_batch_info", load().hx_batch_info(self.handle, ctypes.byref(lt),
                                                     ctypes.byref(tiles), ctypes.byref(launches)))
        return {"limb_transforms": lt.value, "tiles": tiles.value, "launches": launches.value}

    def destroy(self):
        if getattr(self, "handle", None):
            _check("hx_batch_destroy", load().hx_batch_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


# ------------------------------------------------------------- entry points
def hx_ntt_forward(plan, result, operand, n_polys: int, input_mod_factor: int = 1,
                   output_mod_factor: int = 1, stream=None):
    _check("hx_ntt_forward", load().hx_ntt_forward(
        _h(plan), ptr(result), ptr(operand), n_polys, input_mod_factor, output_mod_factor,
        _stream(stream)))


def hx_ntt_inverse(plan, result, operand, n_polys: int, input_mod_factor: int = 1,
                   output_mod_factor: int = 1, stream=None):
    _check("hx_ntt_inverse", load().hx_ntt_inverse(
        _h(plan), ptr(result), ptr(operand), n_polys, input_mod_factor, output_mod_factor,
        _stream(stream)))


def hx_ntt_forward_raw(data, N: int, moduli, input_mod_factor=1, output_mod_factor=1,
                       stream=None):
    _check("hx_ntt_forward_raw", load().hx_ntt_forward_raw(
        ptr(data), N, host_u64(moduli), len(moduli), input_mod_factor, output_mod_factor,
        _stream(stream)))


def hx_ntt_inverse_raw(data, N: int, moduli, input_mod_factor=1, output_mod_factor=1,
                       stream=None):
    _check("hx_ntt_inverse_raw", load().hx_ntt_inverse_raw(
        ptr(data), N, host_u64(moduli), len(moduli), input_mod_factor, output_mod_factor,
        _stream(stream)))


def hx_eltwise_add_mod(result, a, b, n: int, moduli, n_polys: int = 1, stream=None):
    _check("hx_eltwise_add_mod", load().hx_eltwise_add_mod(
        ptr(result), ptr(a), ptr(b), n, host_u64(moduli), len(moduli), n_polys, _stream(stream)))


def hx_eltwise_sub_mod(result, a, b, n: int, moduli, n_polys: int = 1, stream=None):
    _check("hx_eltwise_sub_mod", load().hx_eltwise_sub_mod(
        ptr(result), ptr(a), ptr(b), n, host_u64(moduli), len(moduli), n_polys, _stream(stream)))


def hx_eltwise_negate_mod(result, a, n: int, moduli, n_polys: int = 1, stream=None):
    _check("hx_eltwise_negate_mod", load().hx_eltwise_negate_mod(
        ptr(result), ptr(a), n, host_u64(moduli), len(moduli), n_polys, _stream(stream)))


def hx_eltwise_mult_mod(result, a, b, n: int, moduli, n_polys: int = 1,
                        input_mod_factor: int = 1, stream=None):
    _check("hx_eltwise_mult_mod", load().hx_eltwise_mult_mod(
        ptr(result), ptr(a), ptr(b), n, host_u64(moduli), len(moduli), n_polys,
        input_mod_factor, _stream(stream)))


def hx_eltwise_fma_mod(result, a, scalars, addend, n: int, moduli, n_polys: int = 1,
                       input_mod_factor: int = 1, stream=None):
    _check("hx_eltwise_fma_mod", load().hx_eltwise_fma_mod(
        ptr(result), ptr(a), host_u64(scalars), ptr(addend), n, host_u64(moduli), len(moduli),
        n_polys, input_mod_factor, _stream(stream)))


def hx_poly_mul(plan, result, a, b, n_polys: int, stream=None):
    _check("hx_poly_mul", load().hx_poly_mul(_h(plan), ptr(result), ptr(a), ptr(b), n_polys,
                                             _stream(stream)))


def hx_dyadic_inverse(plan, result, A, B, n_polys: int, input_mod_factor: int = 4,
                      stream=None):
    _check("hx_dyadic_inverse", load().hx_dyadic_inverse(_h(plan), ptr(result), ptr(A), ptr(B),
                                                         n_polys, input_mod_factor,
                                                         _stream(stream)))


def hx_ciphertext_tensor(plan, out0, out1, out2, a0, a1, b0, b1, scalars, e0, e1, e2,
                         n_polys: int, stream=None):
    _check("hx_ciphertext_tensor", load().hx_ciphertext_tensor(
        _h(plan), ptr(out0), ptr(out1), ptr(out2), ptr(a0), ptr(a1), ptr(b0), ptr(b1),
        host_u64(scalars), ptr(e0), ptr(e1), ptr(e2), n_polys, _stream(stream)))


def hx_tensor_fma_inverse(plan, out0, out1, out2, A0, A1, B0, B1, scalars, e0, e1, e2,
                          n_polys: int, input_mod_factor: int = 4, stream=None):
    _check("hx_tensor_fma_inverse", load().hx_tensor_fma_inverse(
        _h(plan), ptr(out0), ptr(out1), ptr(out2), ptr(A0), ptr(A1), ptr(B0), ptr(B1),
        host_u64(scalars), ptr(e0), ptr(e1), ptr(e2), n_polys, input_mod_factor,
        _stream(stream)))


def hx_poly_product(plan, result, a, b, work, n_polys: int = 1, stream=None):
    """result = a * b in R_q, a and b kept; work: [2][n_polys][limbs][N] scratch."""
    _check("hx_poly_product", load().hx_poly_product(
        _h(plan), ptr(result), ptr(a), ptr(b), ptr(work), n_polys, _stream(stream)))


def hx_ciphertext_step(plan, result, inputs, work, scalars, e, n_ct: int, stream=None):
    """result = out0 | out1 | out2 of the ciphertext tensor product of
    inputs = a0 | a1 | b0 | b1 (back to back), addends e = e0 | e1 | e2;
    work is the caller's [4][n_ct][limbs][N] scratch (may be inputs)."""
    _check("hx_ciphertext_step", load().hx_ciphertext_step(
        _h(plan), ptr(result), ptr(inputs), ptr(work), host_u64(scalars), ptr(e), n_ct,
        _stream(stream)))


def hx_dyadic_tensor_fma(r0, r1, r2, A0, A1, B0, B1, scalars, e0, e1, e2, n: int, moduli,
                         n_polys: int = 1, input_mod_factor: int = 1, stream=None):
    _check("hx_dyadic_tensor_fma", load().hx_dyadic_tensor_fma(
        ptr(r0), ptr(r1), ptr(r2), ptr(A0), ptr(A1), ptr(B0), ptr(B1), host_u64(scalars),
        ptr(e0), ptr(e1), ptr(e2), n, host_u64(moduli), len(moduli), n_polys,
        input_mod_factor, _stream(stream)))


def hx_launch_count() -> int:
    return int(load().hx_launch_count())


PROBE_KINDS = {"mad.lo": 0, "mad.hi": 1, "mad.wide": 2, "lo+hi": 3}


def hx_probe_int_mul_rate(kind="mad.lo", iters: int = 4096, stream=None):
    """(32-bit integer multiply instructions per second, kernel ms) of one
    multiply form on the current GPU."""
    r, t = ctypes.c_double(), ctypes.c_float()
    _check("hx_probe_int_mul_rate", load().hx_probe_int_mul_rate(
        PROBE_KINDS.get(kind, kind), iters, ctypes.byref(r), ctypes.byref(t), _stream(stream)))
    return r.value, t.value


def hx_probe_butterfly_rate(q: int, variant: int = 1, inverse: bool = False, iters: int = 4096,
                            stream=None):
    """(Harvey butterflies per second, kernel ms) for modulus q and one
    Shoup-product variant."""
    r, t = ctypes.c_double(), ctypes.c_float()
    _check("hx_probe_butterfly_rate", load().hx_probe_butterfly_rate(
        variant | (16 if inverse else 0), iters, q, ctypes.byref(r), ctypes.byref(t),
        _stream(stream)))
    return r.value, t.value


def hx_probe_copy_rate(dst, src, nbytes: int, iters: int = 10, blocks_per_sm: int = 4,
                       stream=None):
    """(bytes per second, ms per copy) of the library's 16-byte copy kernel
    from src to dst (torch tensors; either may be pinned host memory)."""
    r, t = ctypes.c_double(), ctypes.c_float()
    _check("hx_probe_copy_rate", load().hx_probe_copy_rate(
        ptr(dst), ptr(src), nbytes, iters, blocks_per_sm, ctypes.byref(r), ctypes.byref(t),
        _stream(stream)))
    return r.value, t.value


class LaunchTime(ctypes.Structure):
    """hx_launch_time: one recorded launch."""
    _fields_ = [("kernel", U32), ("reserved", U32), ("ms", ctypes.c_float),
                ("reserved2", ctypes.c_float)]


def hx_timing_enable(on: bool, capacity: int = 0):
    """Start (with room for `capacity` launches) or stop per-launch timing."""
    _check("hx_timing_enable", load().hx_timing_enable(1 if on else 0, capacity))


def hx_timing_read(cap: int = 1 << 16):
    """Recorded launches since the last read, in launch order, as
    (kernel id, ms) pairs; waits for them to finish and clears the record."""
    buf = (LaunchTime * cap)()
    n = U32()
    _check("hx_timing_read", load().hx_timing_read(ctypes.cast(buf, VP), cap, ctypes.byref(n)))
    return [(buf[i].kernel, buf[i].ms) for i in range(n.value)]


def hx_kernel_name(kernel: int) -> str:
    buf = ctypes.create_string_buffer(96)
    _check("hx_kernel_name", load().hx_kernel_name(kernel, buf, 96))
    return buf.value.decode()
