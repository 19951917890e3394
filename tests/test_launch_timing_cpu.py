"""Host side of the per-launch timing (no GPU): kernel ids name the kernels
as CUDA tools print them, nothing is recorded until timing is enabled, and
the bench's per-kernel slot model adds up to the whole-transform model."""
import json

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
    assert capi.hx_kernel_name(kid(2, 0, 0, 3, 9, 0) | 1 << 16) == "ntt_ct_row_kernel<3, 9>"
    assert capi.hx_kernel_name(kid(2, 0, 0, 3, 8, 0) | 3 << 16) == "ntt_mul_row_kernel<3, 8>"
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
    assert all(q < 1 << 61 for q in moduli)
    assert fused - plain == N * (106 * wide + 26 * (len(moduli) - wide))
    # the model from its parts: two Shoup products a s (a butterfly's
    # multiply), three 128-bit products, three Barrett reductions
    prod, red_t, red_x = 4 * 3, 7 + 5, 11 + 5
    assert 2 * bench.SLOTS_WIDE_TRUNC + 3 * prod + 3 * red_t == bench.SLOTS_TENSOR_WIDE_TRUNC
    assert 2 * bench.SLOTS_WIDE + 3 * prod + 3 * red_x == bench.SLOTS_TENSOR_WIDE
    assert 2 * bench.SLOTS_NARROW + 3 * 3 + 3 * (2 + 1) == bench.SLOTS_TENSOR_NARROW
    assert [bench.slots_per_tensor_position(q) for q in ((1 << 30) - 35, 1 << 40, 1 << 61)] \
        == [26, 106, 126]


def test_operation_count_model_at_the_benchmark_size():
    """The operation-count roofline at N = 2^16 x 32 mixed limbs: a forward
    call over 4 polynomials is 16 stages x 32768 butterflies x (21 wide limbs
    x 10 + 11 narrow x 3) x 4 = 509.6 M operations against 134.2 MB (integer
    side slower at 20 T/s and 6786.6 GB/s); the fused tensor / first inverse
    pass (9 stages, 3 outputs) is 215 M operations against 167.8 MB (seven
    operands read, three outputs written): HBM side slower."""
    N, moduli = 1 << 16, W.mixed_width_primes(32)
    assert sum(1 for q in moduli if q < 1 << 30) == 11
    col = bench.kernel_slots(kid(0, 1, 1, 4, 7), N, moduli, per_butterfly=bench.ops_per_butterfly)
    row = bench.kernel_slots(kid(0, 1, 0, 3, 9), N, moduli, per_butterfly=bench.ops_per_butterfly)
    assert col + row == 4 * 16 * 32768 * (21 * 10 + 11 * 3) == 509607936
    clu = bench.kernel_slots(kid(3, 1, 0, 4, 8, 0) | 8 << 15, N, moduli,
                             per_butterfly=bench.ops_per_butterfly)
    assert clu == col + row                      # one cluster launch = the whole transform
    r = bench.op_roofline(col + row, bench.kernel_bytes(kid(3, 1, 0, 4, 8, 0) | 8 << 15, N, 32),
                          91.0, 20.0e12, 6786.6)
    assert r["bound"] == "alu" and abs(r["int_us"] - 25.48) < 0.01
    assert abs(r["hbm_us"] - 134217728 / 6786.6e3) < 1e-9 and abs(r["frac"] - 25.48 / 91) < 1e-3
    fused = kid(2, 0, 0, 3, 9, 3)
    ops = bench.kernel_slots(fused, N, moduli, per_butterfly=bench.ops_per_butterfly)
    assert ops == 3 * 9 * 32768 * (21 * 10 + 11 * 3) == 214990848
    nbytes = bench.kernel_bytes(fused, N, 32)
    assert nbytes == 167772160
    r = bench.op_roofline(ops, nbytes, 69.61, 20.0e12, 6782.0)
    assert r["bound"] == "hbm" and abs(r["frac"] - 0.3554) < 1e-3
    assert abs(r["achieved"] - nbytes / 69.61e-6 / 1e9) < 1e-6 and r["peak"] == 6782.0
    # the cluster tensor launch: all 16 inverse stages plus N^-1, same bytes
    ct = kid(3, 0, 0, 4, 8, 1) | 8 << 15
    assert bench.kernel_bytes(ct, N, 32) == nbytes
    assert (bench.kernel_slots(ct, N, moduli, per_butterfly=bench.ops_per_butterfly)
            == 3 * 17 * 32768 * (21 * 10 + 11 * 3))


def test_traffic_is_reported_only_for_the_captured_sources(monkeypatch):
    h = bench.kernel_source_hash()
    assert len(h) == 16 and h == bench.kernel_source_hash()
    sched = [(0, 8, 0, 3, 4, 0, 1), (8, 8, 1, 0, 3, 0, 1)]
    key = json.dumps([list(p) for p in sched])
    monkeypatch.setattr(bench, "TRAFFIC_BYTES", {("forward_call", key, h): 123,
                                                  ("forward_call", key, "0" * 16): 456})
    assert bench.traffic_for("forward_call", sched) == 123
    monkeypatch.setattr(bench, "TRAFFIC_BYTES", {("forward_call", key, "0" * 16): 456})
    assert bench.traffic_for("forward_call", sched) is None      # other sources: no figure
    assert bench.traffic_for("forward_call", None) is None


def test_forward_inverse_figures():
    """fwd_inv_figures on the benchmark shape: the slot model over both calls
    = (4 forward + 3 inverse transforms' slots) / time / peak; the
    operation count: the forward call is integer-bound (25.5 us at 20 T/s),
    the three-polynomial inverse too (19.1 + 1.2 us of integer work vs 14.8 us
    of HBM at 6786.6 GB/s)."""
    N, moduli = 1 << 16, W.mixed_width_primes(32)
    f = bench.fwd_inv_figures(N, moduli, 90.0, 85.0, 20.0e12, 6786.6)
    slots = 4 * sum(bench.imad_slots_per_transform(N, moduli))
    slots += 3 * (slots // 4 + sum(N // 2 * bench.slots_per_butterfly(q) for q in moduli))
    assert abs(f["fwd_plus_inv_frac_slots"] - slots / 175e-6 / 20e12) < 1e-9
    assert 0.3 < f["fwd_plus_inv_frac_slots"] < 0.6
    ops_f = 4 * 16 * 32768 * (21 * 10 + 11 * 3)
    ops_i = 3 * 17 * 32768 * (21 * 10 + 11 * 3)
    assert f["forward_bound"] == f["inverse_bound"] == "alu"
    assert abs(f["fwd_plus_inv_frac"] - (ops_f + ops_i) / 20e12 / 175e-6) < 1e-9
    assert abs(f["fwd_plus_inv_pairs_per_s"] - 1e6 / (90 / 128 + 85 / 96)) < 1e-6


def test_step_work():
    """One step at 2^16 x 32 mixed limbs: 16 forward stages on 4 polynomials
    and 17 inverse stage-equivalents (N^-1 folded) on 3, 243 operations per
    butterfly column over the limbs (21 x 10 + 11 x 3); 18 polynomial-sized
    HBM transfers (8 for the forward, 10 for tensor + inverse)."""
    N, moduli = 1 << 16, W.mixed_width_primes(32)
    ops, slots, nbytes = bench.step_work(N, moduli)
    assert ops == (4 * 16 + 3 * 17) * 32768 * 243
    assert nbytes == 18 * 8 * N * 32
    tensor = N * (21 * 106 + 11 * 26)
    assert slots == (4 * 16 + 3 * 17) * 32768 * (21 * 17 + 11 * 4) + tensor


def test_step_kernel_work_is_both_row_passes_and_the_tensor():
    """The step kernel (forward row stages on four operands, the tensor, the
    inverse row stages on three outputs): its slots are the forward row
    pass's plus the fused pass's, its bytes the fused pass's (seven operands
    in, three out)."""
    N, moduli = 1 << 16, W.mixed_width_primes(32)
    step = kid(2, 0, 0, 3, 9, 0) | 1 << 16
    fused = bench.kernel_slots(kid(2, 0, 0, 3, 9, 3), N, moduli)
    fwd_row = bench.kernel_slots(kid(0, 1, 0, 3, 9), N, moduli)
    assert bench.kernel_slots(step, N, moduli) == fused + fwd_row
    ops = bench.kernel_slots(step, N, moduli, per_butterfly=bench.ops_per_butterfly)
    assert ops == 7 * 9 * (N // 2) * (21 * 10 + 11 * 3)
    assert bench.kernel_bytes(step, N, 32) == bench.kernel_bytes(kid(2, 0, 0, 3, 9, 3), N, 32)


def test_product_step_kernel_work():
    """The product's step kernel: the forward's row stages on a and b and the
    inverse's on their product (three polynomials' worth of row stages);
    a and b in, a b out."""
    N, moduli = 1 << 16, W.mixed_width_primes(32)
    mul = kid(2, 0, 0, 3, 8, 0) | 3 << 16
    row_inv = bench.kernel_slots(kid(0, 0, 0, 3, 8), N, moduli)       # three polynomials
    assert bench.kernel_slots(mul, N, moduli) == row_inv
    assert bench.kernel_bytes(mul, N, 32) == 3 * 8 * N * 32
