"""hx_poly_product (a * b in R_q with the operands kept: forward NTT of both,
the dyadic product, the inverse NTT) against the oracle's product.  Covers
the four-launch form (the forward's row stages on a and b, the product and
the inverse's row stages in one kernel) under the default schedules at
N = 2^14 .. 2^16, mixed 30/50/60/62-bit limbs, more limbs than 64, the
result written over an operand, the single-pass fallback at N = 2^12, and
argument errors."""
import numpy as np
import pytest

import oracle
import workloads as W
from paper_2103_16400_gb300 import capi
from paper_2103_16400_gb300.tensors import empty, to_device, to_host

pytestmark = pytest.mark.gpu

HX_ERR_OVERLAP = -9   # include/hexgpu.h


def operands(seed, n_polys, moduli, N):
    return (W.poly_batch(seed, 0, n_polys, moduli, N), W.poly_batch(seed, 1, n_polys, moduli, N))


@pytest.mark.parametrize("logN,n_limbs,n_polys,fused", [
    (12, 4, 2, False), (14, 4, 2, True), (15, 5, 1, True), (16, 4, 1, True)])
def test_product_matches_oracle(hexlib, logN, n_limbs, n_polys, fused):
    N = 1 << logN
    moduli = W.mixed_width_primes(n_limbs - 1) + W.mixed_width_primes(1, widths=(62, 62, 62))
    a, b = operands(W.SEED_BASE + 1100 + logN, n_polys, moduli, N)
    plan = capi.Plan(N, moduli)
    da, db = to_device(a), to_device(b)
    R, work = empty(a.shape), empty((2,) + a.shape)
    before = capi.hx_launch_count()
    capi.hx_poly_product(plan, R, da, db, work, n_polys)
    launches = capi.hx_launch_count() - before
    assert launches == (4 if fused else 3)
    np.testing.assert_array_equal(to_host(R), oracle.poly_mul(a, b, moduli))
    np.testing.assert_array_equal(to_host(da), a)       # operands kept
    np.testing.assert_array_equal(to_host(db), b)


def test_result_over_an_operand_and_many_limbs(hexlib):
    N, n_polys = 1 << 14, 1
    moduli = W.mixed_width_primes(70)
    a, b = operands(W.SEED_BASE + 1150, n_polys, moduli, N)
    plan = capi.Plan(N, moduli)
    da, db = to_device(a), to_device(b)
    work = empty((2,) + a.shape)
    capi.hx_poly_product(plan, da, da, db, work, n_polys)      # d_result = d_a
    np.testing.assert_array_equal(to_host(da), oracle.poly_mul(a, b, moduli))
    np.testing.assert_array_equal(to_host(db), b)


def test_rejects_overlapping_buffers(hexlib):
    N, n_polys = 1 << 14, 1
    moduli = W.mixed_width_primes(3)
    plan = capi.Plan(N, moduli)
    a, b = operands(W.SEED_BASE + 1160, n_polys, moduli, N)
    da, db = to_device(a), to_device(b)
    work = empty((2,) + a.shape)
    with pytest.raises(capi.HexError) as ei:             # scratch over an operand
        capi.hx_poly_product(plan, empty(a.shape), da, db, da, n_polys)
    assert ei.value.status == HX_ERR_OVERLAP
    both = empty((2,) + a.shape)
    with pytest.raises(capi.HexError) as ei:             # result partly over an operand
        capi.hx_poly_product(plan, both.view(-1)[N:N + a.size].view(a.shape), both[0], db,
                             work, n_polys)
    assert ei.value.status == HX_ERR_OVERLAP
