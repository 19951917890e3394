"""Cyclic NTT plans (Section 2.2: NTT(a)_i = sum_j a_j omega^(ij), omega a
primitive N-th root) through the C ABI against the oracle's definitions:
forward in bit-reversed order (full at N <= 4096, sampled at 2^16), inverse,
lazy output ranges, the product in Z_q[X] / (X^N - 1) from hx_poly_mul, and
the plan's arguments (q = 1 mod N suffices; the root must have order N)."""
import numpy as np
import pytest

import oracle
import workloads as W
from paper_2103_16400_gb300 import capi
from paper_2103_16400_gb300.capi import HexError, Plan
from paper_2103_16400_gb300.tensors import empty, to_device, to_host

pytestmark = pytest.mark.gpu


def brv_perm(N):
    logn = N.bit_length() - 1
    return np.array([int(format(i, f"0{logn}b")[::-1], 2) for i in range(N)])


def cyclic_ref(x, moduli, roots, idx=None):
    """Bit-reversed cyclic NTT of [n][L][N] (or the outputs at positions idx)."""
    N = x.shape[-1]
    perm = brv_perm(N)
    pos = np.arange(N) if idx is None else np.asarray(idx)
    out = np.empty(x.shape[:2] + (len(pos),), dtype=np.uint64)
    for p in range(x.shape[0]):
        for l, (q, w) in enumerate(zip(moduli, roots)):
            out[p, l] = oracle.cyclic_ntt_1(x[p, l], q, w, perm[pos])
    return out


@pytest.mark.parametrize("logN,n_limbs", [(10, 3), (12, 4)])
def test_cyclic_forward_inverse_full(hexlib, logN, n_limbs):
    N = 1 << logN
    moduli = W.mixed_width_primes(n_limbs)
    plan = Plan(N, moduli, cyclic=True)
    roots = plan.roots()
    assert roots == [oracle.min_primitive_nth_root(N, q) for q in moduli]
    x = W.poly_batch(W.SEED_BASE + 800 + logN, 1, 2, moduli, N, in_mf=4)
    exp = cyclic_ref(x, moduli, roots)
    d, y = to_device(x), empty(x.shape)
    capi.hx_ntt_forward(plan, y, d, 2, 4, 1)
    np.testing.assert_array_equal(to_host(y), exp)
    capi.hx_ntt_forward(plan, y, d, 2, 4, 4)
    lazy = to_host(y)
    for l, q in enumerate(moduli):
        assert (lazy[:, l] < 4 * q).all()
        np.testing.assert_array_equal(lazy[:, l] % np.uint64(q), exp[:, l])
    back = empty(x.shape)
    capi.hx_ntt_forward(plan, y, d, 2, 4, 1)
    capi.hx_ntt_inverse(plan, back, y, 2, 1, 1)
    red = np.stack([x[:, l] % np.uint64(q) for l, q in enumerate(moduli)], axis=1)
    np.testing.assert_array_equal(to_host(back), red)
    # the inverse against its own definition on a random spectrum (natural order)
    z = W.poly_batch(W.SEED_BASE + 820 + logN, 2, 1, moduli, N)
    capi.hx_ntt_inverse(plan, back, to_device(z), 1, 1, 1)
    perm = brv_perm(N)
    got = to_host(back)
    for l, (q, w) in enumerate(zip(moduli, roots)):
        nat = np.empty(N, dtype=np.uint64)
        nat[perm] = z[0, l]                       # input is bit-reversed
        np.testing.assert_array_equal(got[0, l], oracle.cyclic_intt_1(nat, q, w))


def test_cyclic_sampled_n65536(hexlib):
    N = 1 << 16
    moduli = W.mixed_width_primes(6)
    plan = Plan(N, moduli, cyclic=True)
    x = W.poly_batch(W.SEED_BASE + 840, 1, 1, moduli, N)
    d, y = to_device(x), empty(x.shape)
    capi.hx_ntt_forward(plan, y, d, 1, 1, 1)
    idx = [0, 1, 2, 3, 4097, 30000, N // 2, N - 1]
    np.testing.assert_array_equal(to_host(y)[:, :, idx], cyclic_ref(x, moduli, plan.roots(), idx))
    back = empty(x.shape)
    capi.hx_ntt_inverse(plan, back, y, 1, 1, 1)
    np.testing.assert_array_equal(to_host(back), x)


def test_cyclic_polymul_is_cyclic_convolution(hexlib):
    N = 1 << 11
    moduli = W.mixed_width_primes(3)
    plan = Plan(N, moduli, cyclic=True)
    a = W.poly_batch(W.SEED_BASE + 860, 1, 1, moduli, N)
    b = W.poly_batch(W.SEED_BASE + 860, 2, 1, moduli, N)
    da, db, dr = to_device(a), to_device(b), empty(a.shape)
    capi.hx_poly_mul(plan, dr, da, db, 1)
    got = to_host(dr)
    for l, q in enumerate(moduli):
        np.testing.assert_array_equal(got[0, l], oracle.cyclic_schoolbook(a[0, l], b[0, l], q))


def test_cyclic_plan_arguments(hexlib):
    N = 1 << 10
    # q = 1 mod N but not mod 2N: fine for the cyclic transform only
    q = next(c for c in range(N + 1, 1 << 40, N) if c % (2 * N) != 1 and W.is_prime(c))
    Plan(N, [q], cyclic=True)
    with pytest.raises(HexError):
        Plan(N, [q])
    qs = list(W.ntt_primes(50, 2 * N, 1))
    w = oracle.min_primitive_nth_root(N, qs[0])
    Plan(N, qs, roots=[w], cyclic=True)
    with pytest.raises(HexError):                    # order N/2, not N
        Plan(N, qs, roots=[w * w % qs[0]], cyclic=True)
    psi = oracle.min_primitive_root(N, qs[0])
    with pytest.raises(HexError):                    # order 2N, not N
        Plan(N, qs, roots=[psi], cyclic=True)
    x = W.poly_batch(W.SEED_BASE + 880, 1, 1, qs, N)
    plan = Plan(N, qs, roots=[oracle.invmod(w, qs[0])], cyclic=True)   # another primitive root
    y = empty(x.shape)
    capi.hx_ntt_forward(plan, y, to_device(x), 1, 1, 1)
    np.testing.assert_array_equal(to_host(y), cyclic_ref(x, qs, [oracle.invmod(w, qs[0])]))
