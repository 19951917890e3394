"""Host side of the per-launch timing (no GPU): kernel ids name the kernels
as CUDA tools print them, nothing is recorded until timing is enabled, and
the bench's per-kernel slot model adds up to the whole-transform model."""
import pytest

import bench
import workloads as W
from paper_2103_16400_gb300 import capi


def kid(kind, fwd=0, column=0, logR=3, K=8, np_=1, tws=0):
    return kind | fwd << 2 | column << 3 | logR << 4 | K << 7 | np_ << 12 | tws << 14


def test_kernel_names():
    assert capi.hx_kernel_name(kid(0, 1, 1, 4, 8)) == "ntt_pass_kernel<1, 1, 4, 8, 1, 0>"
    assert capi.hx_kernel_name(kid(0, 0, 1, 4, 7, 1, 1)) == "ntt_pass_kernel<0, 1, 4, 7, 1, 1>"
    assert capi.hx_kernel_name(kid(1, 1, 0, 3, 9)) == "ntt_pipe_kernel<1, 0, 3, 9>"
    assert capi.hx_kernel_name(kid(2, 0, 0, 3, 9, 3)) == "ntt_tensor_inv_kernel<3, 9, 0, 3>"
    # cluster-fused transforms: kind 3, K1 in the K field, K2 in bits 15-19
    assert capi.hx_kernel_name(kid(3, 1, 0, 4, 8, 0) | 8 << 15) == "ntt_cluster_kernel<1, 4, 8, 8>"
    assert (capi.hx_kernel_name(kid(3, 0, 0, 4, 7, 1) | 9 << 15)
            == "ntt_cluster_tensor_kernel<4, 7, 9>")


def test_nothing_recorded_while_off():
    assert capi.hx_timing_read(8) == []
    with pytest.raises(capi.HexError):
        capi.hx_timing_enable(True, 0)          # capacity must be 1 .. 2^20


@pytest.mark.parametrize("logN,K1", [(16, 7), (16, 8), (14, 6)])
def test_pass_slots_add_up_to_the_transform(logN, K1):
    N = 1 << logN
    moduli = W.mixed_width_primes(32)
    col = bench.kernel_slots(kid(0, 1, 1, 4, K1), N, moduli)
    row = bench.kernel_slots(kid(0, 1, 0, 3, logN - K1), N, moduli)
    assert col + row == 4 * sum(bench.imad_slots_per_transform(N, moduli))
    inv = bench.kernel_slots(kid(0, 0, 1, 4, K1), N, moduli)
    # three polynomials in the inverse, whose last stage also scales by N^-1
    scale = 3 * sum(N // 2 * bench.slots_per_butterfly(q) for q in moduli)
    assert (inv - scale) * 4 == col * 3
    assert bench.kernel_slots(kid(0, 0, 0, 3, logN - K1), N, moduli) * 4 == row * 3


def test_fused_slots_are_butterflies_plus_the_tensor_step():
    N, moduli = 1 << 16, W.mixed_width_primes(32)
    fused = bench.kernel_slots(kid(2, 0, 0, 3, 9, 3), N, moduli)
    plain = bench.kernel_slots(kid(0, 0, 0, 3, 9), N, moduli)
    wide = sum(1 for q in moduli if q >= 1 << 30)
    assert fused - plain == N * (175 * wide + 33 * (len(moduli) - wide))
    # the element-wise model from its parts: products, reductions, FMAs
    mul_w, red_w, fma_w = 11 + 5, 11 + 5, 5 + 11 + 5
    assert (mul_w + red_w) * 2 + (2 * mul_w + red_w) + 3 * fma_w == bench.SLOTS_TENSOR_WIDE
    mul_n, red_n, fma_n = 3, 2 + 1, 1 + 2 + 1
    assert (mul_n + red_n) * 2 + (2 * mul_n + red_n) + 3 * fma_n == bench.SLOTS_TENSOR_NARROW
