"""Host logic of the ragged-product binding (no GPU): the item array a server
builds column by column in numpy holds the same bytes as the ctypes array of
hx_polymul_item, and a malformed array is refused before any call."""
import ctypes

import numpy as np
import pytest

from paper_2103_16400_gb300 import capi


def test_numpy_items_match_ctypes_items():
    plans = [0x7f0000001000, 0x7f0000002000, 0x7f0000001000]
    a = [0x7e0000000000 + 4096 * i for i in range(3)]
    b = [0x7d0000000000 + 8192 * i for i in range(3)]
    r = np.array([0x7c0000000000, 0x7c0000100000, 0x7c0000300000], np.int64)
    arr, n = capi.polymul_items_array(plans, a, b, r, [1, 2, 3])
    ref, n_ref = capi.polymul_items(list(zip(plans, a, b, [int(x) for x in r], [1, 2, 3])))
    assert n == n_ref == 3
    assert arr.tobytes() == bytes(ref)
    assert capi._items_ptr(arr).value == arr.ctypes.data
    assert capi._items_ptr(ref).value == ctypes.addressof(ref)


def test_malformed_item_arrays_are_refused():
    arr, _ = capi.polymul_items_array([1, 2, 3], [3, 4, 5], [5, 6, 7], [7, 8, 9])
    with pytest.raises(ValueError):
        capi._items_ptr(arr[::2])                      # not contiguous
    with pytest.raises(ValueError):
        capi._items_ptr(np.zeros(2, np.uint64))        # not an item array


def test_numpy_ragged_items_match_ctypes_items():
    plans = [0x7f0000001000, 0x7f0000002000]
    i = [0x7e0000000000, 0x7e0000010000]
    o = np.array([0x7c0000000000, 0x7c0000100000], np.int64)
    arr, n = capi.ragged_items_array(plans, i, o, [1, 3])
    p, n2, keep = capi._ragged_ptr((arr, n))
    assert n == n2 == 2 and p.value == arr.ctypes.data and keep is arr
    p_ref, n_ref, ref = capi._ragged_ptr(list(zip(plans, i, [int(x) for x in o], [1, 3])))
    assert n_ref == 2 and arr.tobytes() == bytes(ref)
    with pytest.raises(ValueError):
        capi._ragged_ptr((np.zeros(2, np.uint64), 2))
