"""Parity of the CUDA element-wise kernels and compositions (through the C
ABI) with the CPU oracle: bit-exact, ragged lengths, lazy input ranges,
more limbs than one launch takes, and the full workload shapes (one
polynomial multiply at N=1024, the 8-limb RNS multiply at N=16384 and the
ciphertext tensor product at N=32768 and 65536 with 32 mixed limbs)."""
import numpy as np
import pytest

import oracle
import workloads as W
from paper_2103_16400_gb300 import capi
from paper_2103_16400_gb300.capi import HexError, Plan
from paper_2103_16400_gb300.tensors import empty, to_device, to_host

pytestmark = pytest.mark.gpu


def rows(seed, tag, n_polys, moduli, n, in_mf=1):
    return W.poly_batch(seed, tag, n_polys, moduli, n, in_mf=in_mf)


ELT_CASES = [  # (n, n_polys, moduli)
    (1, 1, [3]),
    (7, 2, [97, (1 << 61) - 1]),
    (1024, 1, list(W.ntt_primes(50, 2048, 1))),
    (4099, 3, W.mixed_width_primes(5)),
    (65536, 2, W.mixed_width_primes(70)),      # more limbs than one launch holds
]


@pytest.mark.parametrize("n,n_polys,moduli", ELT_CASES)
def test_add_sub(hexlib, n, n_polys, moduli):
    a, b = rows(1, 1, n_polys, moduli, n), rows(1, 2, n_polys, moduli, n)
    da, db, dr = to_device(a), to_device(b), empty(a.shape)
    capi.hx_eltwise_add_mod(dr, da, db, n, moduli, n_polys)
    np.testing.assert_array_equal(to_host(dr), oracle.eltwise_add_mod(a, b, moduli))
    capi.hx_eltwise_sub_mod(dr, da, db, n, moduli, n_polys)
    exp = np.empty_like(a)
    for p in range(n_polys):
        for l, q in enumerate(moduli):
            exp[p, l] = oracle.eltwise_sub_mod_1(a[p, l], b[p, l], q)
    np.testing.assert_array_equal(to_host(dr), exp)


@pytest.mark.parametrize("n,n_polys,moduli", ELT_CASES)
@pytest.mark.parametrize("in_mf", [1, 2, 4])
def test_mult(hexlib, n, n_polys, moduli, in_mf):
    moduli = [q for q in moduli if q < (1 << 61)] or [3]
    a = rows(2, 1, n_polys, moduli, n, in_mf)
    b = rows(2, 2, n_polys, moduli, n, in_mf)
    da, db, dr = to_device(a), to_device(b), empty(a.shape)
    capi.hx_eltwise_mult_mod(dr, da, db, n, moduli, n_polys, in_mf)
    np.testing.assert_array_equal(to_host(dr), oracle.eltwise_mult_mod(a, b, moduli))
    capi.hx_eltwise_mult_mod(da, da, db, n, moduli, n_polys, in_mf)     # in place
    np.testing.assert_array_equal(to_host(da), oracle.eltwise_mult_mod(a, b, moduli))


def test_mult_barrett_edges(hexlib):
    """q just above a power of two, and 59..62-bit q, with operands q-1, q-2
    (where the Barrett estimate falls short by two)."""
    moduli = [(1 << 29) + 11, (1 << 49) + 9, (1 << 58) + 27, (1 << 59) + 21, (1 << 60) + 33,
              (1 << 61) + 15, (1 << 62) - 57, (1 << 62) - 87]
    n = 64
    a = np.zeros((1, len(moduli), n), dtype=np.uint64)
    b = np.zeros_like(a)
    for l, q in enumerate(moduli):
        vals = [q - 1, q - 2, q // 2, 1, 0, q - 3, (q + 1) // 2, q - 1] * 8
        a[0, l] = vals
        b[0, l] = vals[::-1]
    dr = empty(a.shape)
    capi.hx_eltwise_mult_mod(dr, to_device(a), to_device(b), n, moduli, 1, 1)
    np.testing.assert_array_equal(to_host(dr), oracle.eltwise_mult_mod(a, b, moduli))


@pytest.mark.parametrize("n,n_polys,moduli", ELT_CASES)
@pytest.mark.parametrize("in_mf", [1, 8])
@pytest.mark.parametrize("with_addend", [True, False])
def test_fma(hexlib, n, n_polys, moduli, in_mf, with_addend):
    moduli = [q for q in moduli if q < (1 << 61)] or [3]
    a = rows(3, 1, n_polys, moduli, n, in_mf)
    d = rows(3, 2, n_polys, moduli, n, in_mf) if with_addend else None
    s = W.scalars(3, 3, moduli)
    da, dr = to_device(a), empty(a.shape)
    dd = to_device(d) if with_addend else None
    capi.hx_eltwise_fma_mod(dr, da, s, dd, n, moduli, n_polys, in_mf)
    np.testing.assert_array_equal(to_host(dr), oracle.eltwise_fma_mod(a, s, d, moduli))


def test_argument_errors(hexlib):
    moduli = [97]
    a = to_device(np.zeros((1, 1, 8), dtype=np.uint64))
    with pytest.raises(HexError) as e:
        capi.hx_eltwise_mult_mod(a, a, a, 8, moduli, 1, 3)
    assert e.value.status == -6
    with pytest.raises(HexError) as e:
        capi.hx_eltwise_add_mod(a.data_ptr() + 8, a, a, 8, moduli, 1)
    assert e.value.status == -2
    with pytest.raises(HexError) as e:
        capi.hx_eltwise_fma_mod(a, a, [97], None, 8, moduli, 1, 1)     # scalar >= q
    assert e.value.status == -8
    plan = Plan(1024, list(W.ntt_primes(50, 2048, 1)))
    buf = empty((1, 1, 1024))
    with pytest.raises(HexError) as e:
        capi.hx_ntt_forward(plan, buf, buf, 1, 1, 2)                   # out_mf 2 not allowed
    assert e.value.status == -6
    with pytest.raises(HexError) as e:
        capi.hx_ntt_inverse(plan, buf.data_ptr() + 16, buf, 1, 1, 1)   # partial overlap
    assert e.value.status == -9


# ------------------------------------------------------------ compositions
def test_single_polymul_n1024_against_schoolbook(hexlib):
    wl = W.single_ntt_1024()
    q = wl.moduli[0]
    a = rows(wl.seed, 1, 1, wl.moduli, wl.N)
    b = rows(wl.seed, 2, 1, wl.moduli, wl.N)
    plan = Plan(wl.N, wl.moduli)
    da, db, dr = to_device(a), to_device(b), empty(a.shape)
    capi.hx_poly_mul(plan, dr, da, db, 1)
    got = to_host(dr)[0, 0]
    np.testing.assert_array_equal(got, oracle.negacyclic_schoolbook(a[0, 0], b[0, 0], q))
    # the forward transforms left in the operands are the lazy [0, 4q) NTTs
    assert_fa = to_host(da)[0, 0]
    assert (assert_fa < np.uint64(4 * q)).all()
    np.testing.assert_array_equal(assert_fa % np.uint64(q), oracle.ntt_forward_1(a[0, 0], q))


def test_rns_polymul_n16384(hexlib):
    wl = W.rns_polymul_16384()
    a = rows(wl.seed, 1, 2, wl.moduli, wl.N)
    b = rows(wl.seed, 2, 2, wl.moduli, wl.N)
    plan = Plan(wl.N, wl.moduli)
    da, db = to_device(a), to_device(b)
    capi.hx_poly_mul(plan, da, da, db, 2)                # result over operand a
    got = to_host(da)
    np.testing.assert_array_equal(got, oracle.poly_mul(a, b, wl.moduli))
    idx = [0, 1, 8191, 16383]                            # brute-force spot checks
    for l, q in enumerate(wl.moduli):
        np.testing.assert_array_equal(got[1, l, idx],
                                      oracle.negacyclic_schoolbook(a[1, l], b[1, l], q, idx))


@pytest.mark.parametrize("N", [1 << 15, 1 << 16])
def test_ciphertext_tensor_full(hexlib, N):
    wl = W.ciphertext_tensor(N=N)
    qs = wl.moduli
    ins = [rows(wl.seed, t, 1, qs, N) for t in range(4)]
    es = [rows(wl.seed, 10 + t, 1, qs, N) for t in range(3)]
    s = W.scalars(wl.seed, 20, qs)
    plan = Plan(N, qs)
    d_ins = [to_device(x) for x in ins]
    d_es = [to_device(x) for x in es]
    outs = [empty(ins[0].shape) for _ in range(3)]
    capi.hx_ciphertext_tensor(plan, *outs, *d_ins, s, *d_es, 1)
    exp = oracle.ciphertext_tensor(*ins, s, *es, qs)
    for o, e in zip(outs, exp):
        np.testing.assert_array_equal(to_host(o), e)


def test_dyadic_tensor_fma_lazy_inputs(hexlib):
    n, qs = 4096 + 6, W.mixed_width_primes(4)
    A = [rows(7, t, 2, qs, n, in_mf=4) for t in range(4)]
    E = [rows(7, 10 + t, 2, qs, n) for t in range(3)]
    s = W.scalars(7, 20, qs)
    outs = [empty(A[0].shape) for _ in range(3)]
    capi.hx_dyadic_tensor_fma(*outs, *[to_device(x) for x in A], s,
                              *[to_device(x) for x in E], n, qs, 2, 4)
    a0, a1, b0, b1 = A
    M = lambda x, y: oracle.eltwise_mult_mod(x, y, qs)
    d = [M(a0, b0), oracle.eltwise_add_mod(M(a0, b1), M(a1, b0), qs), M(a1, b1)]
    for o, dk, ek in zip(outs, d, E):
        np.testing.assert_array_equal(to_host(o), oracle.eltwise_fma_mod(dk, s, ek, qs))


@pytest.mark.parametrize("n,n_polys,moduli", ELT_CASES)
def test_negate(hexlib, n, n_polys, moduli):
    """(q - a) mod q, with zeros planted (they must stay 0), out of place and
    in place."""
    a = rows(1, 3, n_polys, moduli, n)
    a[:, :, ::5] = 0
    exp = oracle.eltwise_negate_mod(a, moduli)
    da, dr = to_device(a), empty(a.shape)
    capi.hx_eltwise_negate_mod(dr, da, n, moduli, n_polys)
    np.testing.assert_array_equal(to_host(dr), exp)
    capi.hx_eltwise_negate_mod(da, da, n, moduli, n_polys)
    np.testing.assert_array_equal(to_host(da), exp)
