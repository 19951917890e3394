"""Parity of the CUDA transforms (through the C ABI) with the CPU oracle.

Bit-exact comparison on canonical outputs (output_mod_factor 1); for lazy
outputs (factor 2 or 4) every value must lie in [0, factor*q) and be
congruent mod q to the oracle's value, the only thing the paper fixes for
them (Section 3, NTT class API).  Sizes span every N from 2^10 to 2^17
with 30-, 50- and 60-bit primes and several polynomials per call."""
import numpy as np
import pytest

import oracle
import workloads as W
from paper_2103_16400_gb300 import capi
from paper_2103_16400_gb300.capi import Plan
from paper_2103_16400_gb300.tensors import empty, to_device, to_host

pytestmark = pytest.mark.gpu

MIXED3 = W.mixed_width_primes(3)   # one 30-, one 50-, one 60-bit prime, = 1 mod 2^18


def assert_lazy(got, exp, moduli, factor):
    for l, q in enumerate(moduli):
        g, e = got[:, l], exp[:, l]
        assert (g < np.uint64(factor * q)).all(), f"limb {l}: value >= {factor}q"
        np.testing.assert_array_equal(g % np.uint64(q), e)


def gpu_forward(plan, x, in_mf=1, out_mf=1, inplace=False):
    d = to_device(x)
    out = d if inplace else empty(d.shape)
    capi.hx_ntt_forward(plan, out, d, x.shape[0], in_mf, out_mf)
    return to_host(out), to_host(d)


def gpu_inverse(plan, x, in_mf=1, out_mf=1, inplace=False):
    d = to_device(x)
    out = d if inplace else empty(d.shape)
    capi.hx_ntt_inverse(plan, out, d, x.shape[0], in_mf, out_mf)
    return to_host(out), to_host(d)


def test_plan_roots_match_oracle(hexlib):
    for N, qs in [(1024, W.ntt_primes(50, 2048, 1)), (1 << 16, MIXED3), (1 << 17, MIXED3)]:
        p = Plan(N, qs)
        assert p.roots() == [oracle.min_primitive_root(N, q) for q in qs]
        N_, nl, nbytes = p.info()
        assert (N_, nl) == (N, len(qs)) and nbytes >= 32 * N * len(qs)


@pytest.mark.parametrize("logN", list(range(10, 18)))
def test_forward_inverse_every_size(hexlib, logN):
    N = 1 << logN
    x = W.poly_batch(W.SEED_BASE + 100 + logN, 1, 2, MIXED3, N)
    plan = Plan(N, MIXED3)
    exp = oracle.ntt_forward(x, MIXED3)
    got, src = gpu_forward(plan, x)
    np.testing.assert_array_equal(got, exp)
    np.testing.assert_array_equal(src, x)            # out-of-place leaves the operand
    lazy, _ = gpu_forward(plan, x, out_mf=4)
    assert_lazy(lazy, exp, MIXED3, 4)
    back, _ = gpu_inverse(plan, got)
    np.testing.assert_array_equal(back, x)
    back2, _ = gpu_inverse(plan, got, out_mf=2, inplace=True)
    assert_lazy(back2, x, MIXED3, 2)


@pytest.mark.parametrize("logN", [10, 13, 14, 16, 17])
def test_inverse_matches_oracle_on_random_spectra(hexlib, logN):
    N = 1 << logN
    y = W.poly_batch(W.SEED_BASE + 200 + logN, 2, 2, MIXED3, N)
    plan = Plan(N, MIXED3)
    got, _ = gpu_inverse(plan, y, inplace=True)
    np.testing.assert_array_equal(got, oracle.ntt_inverse(y, MIXED3))


@pytest.mark.parametrize("logN", [10, 12, 15, 16])
@pytest.mark.parametrize("in_mf", [2, 4])
def test_forward_lazy_inputs(hexlib, logN, in_mf):
    N = 1 << logN
    x = W.poly_batch(W.SEED_BASE + 300 + logN, 3, 1, MIXED3, N, in_mf=in_mf)
    assert any((x[0, l] >= np.uint64(q)).any() for l, q in enumerate(MIXED3))
    plan = Plan(N, MIXED3)
    got, _ = gpu_forward(plan, x, in_mf=in_mf, out_mf=1)
    np.testing.assert_array_equal(got, oracle.ntt_forward(x, MIXED3))


@pytest.mark.parametrize("logN", [11, 16])
def test_inverse_lazy_inputs(hexlib, logN):
    N = 1 << logN
    y = W.poly_batch(W.SEED_BASE + 400 + logN, 4, 2, MIXED3, N, in_mf=2)
    plan = Plan(N, MIXED3)
    got, _ = gpu_inverse(plan, y, in_mf=2, out_mf=1)
    np.testing.assert_array_equal(got, oracle.ntt_inverse(y, MIXED3))


def test_extreme_inputs(hexlib):
    """All coefficients at the top of the allowed range, zeros, and a delta."""
    N = 1 << 14
    qs = MIXED3 + list(W.ntt_primes(61, 1 << 15, 1)) + [W.ntt_primes(62, 1 << 15, 1)[0]]
    plan = Plan(N, qs)
    top = np.stack([np.full(N, 4 * q - 1, dtype=np.uint64) for q in qs])[None]
    got, _ = gpu_forward(plan, top, in_mf=4)
    np.testing.assert_array_equal(got, oracle.ntt_forward(top, qs))
    top2 = np.stack([np.full(N, 2 * q - 1, dtype=np.uint64) for q in qs])[None]
    got, _ = gpu_inverse(plan, top2, in_mf=2)
    np.testing.assert_array_equal(got, oracle.ntt_inverse(top2, qs))
    zero = np.zeros((1, len(qs), N), dtype=np.uint64)
    assert not gpu_forward(plan, zero)[0].any()
    delta = zero.copy(); delta[0, :, 0] = 1
    assert (gpu_forward(plan, delta)[0] == 1).all()          # NTT(1) = (1, ..., 1)


def _largest_ntt_prime_below(bound, two_n):
    q = (bound - 1) // two_n * two_n + 1
    while not W.is_prime(q):
        q -= two_n
    return q


def test_truncated_quotient_boundary(hexlib):
    """64-bit limbs with q < 2^61 take the truncated-quotient Shoup product
    (lazy bound 4q), q >= 2^61 the exact one (2q): the largest NTT prime below
    2^61 and the smallest above (and likewise around 2^60 and 2^50), with
    every coefficient at the top of the allowed input range and with random
    inputs, forward and inverse, canonical and lazy outputs."""
    N = 1 << 13
    qs = [_largest_ntt_prime_below(1 << 61, 2 * N), W.ntt_primes(62, 2 * N, 1)[0],
          _largest_ntt_prime_below(1 << 60, 2 * N), W.ntt_primes(61, 2 * N, 1)[0],
          _largest_ntt_prime_below(1 << 50, 2 * N), MIXED3[2]]
    assert qs[0] < (1 << 61) <= qs[1] and qs[2] < (1 << 60) <= qs[3]
    plan = Plan(N, qs)
    top = np.stack([np.full(N, 4 * q - 1, dtype=np.uint64) for q in qs])[None]
    rnd = W.poly_batch(W.SEED_BASE + 520, 1, 3, qs, N)
    for x, in_mf in ((top, 4), (rnd, 1)):
        exp = oracle.ntt_forward(x, qs)
        got, _ = gpu_forward(plan, x, in_mf=in_mf, out_mf=1)
        np.testing.assert_array_equal(got, exp)
        lazy, _ = gpu_forward(plan, x, in_mf=in_mf, out_mf=4)
        assert_lazy(lazy, exp, qs, 4)
    top2 = np.stack([np.full(N, 2 * q - 1, dtype=np.uint64) for q in qs])[None]
    for y, in_mf in ((top2, 2), (oracle.ntt_forward(rnd, qs), 1)):
        exp = oracle.ntt_inverse(y, qs)
        got, _ = gpu_inverse(plan, y, in_mf=in_mf, out_mf=1)
        np.testing.assert_array_equal(got, exp)
        lazy, _ = gpu_inverse(plan, y, in_mf=in_mf, out_mf=2)
        assert_lazy(lazy, exp, qs, 2)


def test_many_polys_and_limbs(hexlib):
    N = 1 << 10
    qs = W.mixed_width_primes(7)
    x = W.poly_batch(W.SEED_BASE + 500, 5, 37, qs, N)
    plan = Plan(N, qs)
    got, _ = gpu_forward(plan, x)
    np.testing.assert_array_equal(got, oracle.ntt_forward(x, qs))


def test_user_supplied_roots(hexlib):
    N, q = 1 << 12, W.ntt_primes(60, 1 << 13, 1)[0]
    psi = oracle.min_primitive_root(N, q)
    other = oracle.powmod(psi, 3, q)                 # another primitive 2N-th root
    plan = Plan(N, [q], roots=[other])
    assert plan.roots() == [other]
    x = W.poly_batch(W.SEED_BASE + 600, 5, 1, [q], N)
    got, _ = gpu_forward(plan, x)
    exp = oracle.ntt_forward_1(x[0, 0], q, psi=other)
    np.testing.assert_array_equal(got[0, 0], exp)


def test_raw_entry_points_in_place(hexlib):
    N = 1 << 13
    qs = list(W.ntt_primes(50, 2 * N, 2))
    x = W.poly_batch(W.SEED_BASE + 700, 6, 1, qs, N)
    d = to_device(x[0])
    capi.hx_ntt_forward_raw(d, N, qs, 1, 1)
    np.testing.assert_array_equal(to_host(d), oracle.ntt_forward(x, qs)[0])
    capi.hx_ntt_inverse_raw(d, N, qs, 1, 1)
    np.testing.assert_array_equal(to_host(d), x[0])
