"""Per-launch timing through the C ABI: with timing on, every NTT pass and
fused tensor pass of a forward call and a tensor + inverse call leaves one
record (kernel name as CUDA tools print it, positive duration), as many as
the launch counter counted; with timing off nothing is recorded; the
results do not change."""
import numpy as np
import pytest

import oracle
import workloads as W
from paper_2103_16400_gb300 import capi
from paper_2103_16400_gb300.tensors import empty, to_device, to_host

pytestmark = pytest.mark.gpu


def test_records_match_launches(hexlib):
    N = 1 << 14
    moduli = W.mixed_width_primes(6)
    plan = capi.Plan(N, moduli)
    plan.set_schedule([(0, 7, 0, 4, 4, 0, 1), (7, 7, 1, 0, 3, 0, 2)])
    x = W.poly_batch(W.SEED_BASE + 970, 1, 4, moduli, N)
    E = np.stack([W.poly_batch(W.SEED_BASE + 971, t, 1, moduli, N) for t in range(3)])
    s = W.scalars(W.SEED_BASE + 972, 20, moduli)
    dA, dE = to_device(x), to_device(E)
    R = empty((3, 1, len(moduli), N))

    def step():
        capi.hx_ntt_forward(plan, dA, to_device(x), 4, 1, 4)
        capi.hx_tensor_fma_inverse(plan, R[0], R[1], R[2], dA[0:1], dA[1:2], dA[2:3], dA[3:4],
                                   s, dE[0], dE[1], dE[2], 1, 4)

    step()
    ref = to_host(R)
    capi.hx_timing_read(64)
    capi.hx_timing_enable(True, 64)
    n0 = capi.hx_launch_count()
    step()
    step()
    n = capi.hx_launch_count() - n0
    capi.hx_timing_enable(False)
    recs = capi.hx_timing_read(64)
    assert len(recs) == n == 8                    # 2 forward passes + fused + last inverse pass
    names = [capi.hx_kernel_name(k) for k, _ in recs]
    # passes are (s0, K, logGb, logGc, logR, pipe, np): the row pass runs two
    # polynomials a thread, so the fused pass computes all three outputs a block
    assert names[:4] == ["ntt_pass_kernel<1, 1, 4, 7, 1, 0>", "ntt_pass_kernel<1, 0, 3, 7, 2, 0>",
                         "ntt_tensor_inv_kernel<3, 7, 0, 3>", "ntt_pass_kernel<0, 1, 4, 7, 1, 0>"]
    assert names[4:] == names[:4]
    assert all(ms > 0 for _, ms in recs)
    np.testing.assert_array_equal(to_host(R), ref)
    step()                                        # off: nothing recorded
    assert capi.hx_timing_read(64) == []
    # and the product is the oracle's
    exp0 = oracle.ntt_inverse(oracle.eltwise_fma_mod(
        oracle.eltwise_mult_mod(oracle.ntt_forward(x[0:1], moduli),
                                oracle.ntt_forward(x[2:3], moduli), moduli),
        s, E[0], moduli), moduli)
    np.testing.assert_array_equal(ref[0], exp0)
