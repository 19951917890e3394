"""hx_ciphertext_step (the whole ciphertext tensor product from coefficient
form: forward NTT of a0, a1, b0, b1, d0 = A0 B0, d1 = A0 B1 + A1 B0,
d2 = A1 B1, r_k = d_k s + e_k, out_k = InvNTT(r_k)) against the oracle's
composition of the same steps.  Covers the three-launch form (the forward's
row stages, the tensor and the inverse's row stages in one kernel) under
every row tile it takes at N = 2^14 .. 2^16, more limbs than one launch
holds, the operands transformed in place (work = inputs), the fallback to
hx_ntt_forward + hx_tensor_fma_inverse when the two schedules' row passes
differ, and argument errors."""
import numpy as np
import pytest

import oracle
import workloads as W
from paper_2103_16400_gb300 import capi
from paper_2103_16400_gb300.tensors import empty, to_device, to_host

pytestmark = pytest.mark.gpu


def inputs(seed, n_ct, moduli, N):
    ins = np.stack([W.poly_batch(seed, t, n_ct, moduli, N) for t in range(4)])
    es = np.stack([W.poly_batch(seed, 10 + t, n_ct, moduli, N) for t in range(3)])
    return ins, es, W.scalars(seed, 20, moduli)


def expected(ins, es, s, moduli):
    return oracle.ciphertext_tensor(ins[0], ins[1], ins[2], ins[3], s, es[0], es[1], es[2],
                                    moduli)


def run(plan, ins, es, s, n_ct, in_place=False):
    d_in, d_e = to_device(ins), to_device(es)
    work = d_in if in_place else empty(ins.shape)
    R = empty((3,) + ins.shape[1:])
    before = capi.hx_launch_count()
    capi.hx_ciphertext_step(plan, R, d_in, work, s, d_e, n_ct)
    launches = capi.hx_launch_count() - before
    return [to_host(R[k]) for k in range(3)], launches


def step_schedules(logN, K1, logGb, inv_pipe=0, inv_np=2):
    K2 = logN - K1
    fwd = [(0, K1, 0, 4, 4, 0, 1), (K1, K2, logGb, 0, 3, 0, 1)]
    inv = [(0, K1, 0, 4, 4, inv_pipe, 1), (K1, K2, logGb, 0, 3, 0, inv_np)]
    return fwd, inv


@pytest.mark.parametrize("logN,K1,logGb,n_limbs,n_ct", [
    (14, 7, 1, 6, 2), (14, 8, 2, 4, 1), (15, 7, 1, 5, 1), (15, 6, 0, 3, 2),
    (16, 7, 0, 4, 1), (16, 8, 2, 3, 1), (16, 7, 1, 6, 1)])
def test_three_launch_step_matches_oracle(hexlib, logN, K1, logGb, n_limbs, n_ct):
    N = 1 << logN
    moduli = W.mixed_width_primes(n_limbs)
    ins, es, s = inputs(W.SEED_BASE + 900 + logN + K1, n_ct, moduli, N)
    plan = capi.Plan(N, moduli)
    fwd, inv = step_schedules(logN, K1, logGb, inv_pipe=2 if logGb == 0 else 0)
    plan.set_schedule(fwd, plan.FORWARD)
    plan.set_schedule(inv, plan.INVERSE)
    got, launches = run(plan, ins, es, s, n_ct)
    assert launches == 3                      # column, fused rows + tensor, column
    for g, e in zip(got, expected(ins, es, s, moduli)):
        np.testing.assert_array_equal(g, e)


def test_default_schedules_take_the_three_launch_form(hexlib):
    """The plan's default schedules at N = 2^16 have row passes over the same
    stages in different row tiles (forward one row, inverse two): the step
    kernel runs both in the inverse's tiles."""
    N, n_ct = 1 << 16, 1
    moduli = W.mixed_width_primes(4)
    ins, es, s = inputs(W.SEED_BASE + 940, n_ct, moduli, N)
    plan = capi.Plan(N, moduli)
    f, i = plan.schedule(plan.FORWARD), plan.schedule(plan.INVERSE)
    assert f[1][:2] == i[1][:2] and f[1][2] != i[1][2]
    got, launches = run(plan, ins, es, s, n_ct)
    assert launches == 3
    for g, e in zip(got, expected(ins, es, s, moduli)):
        np.testing.assert_array_equal(g, e)


def test_in_place_and_many_limbs(hexlib):
    """70 limbs (two launches of the fused kernel) with the operands
    transformed in place; the inputs are then the forward column pass's
    output, the results unchanged."""
    N, n_ct = 1 << 14, 1
    moduli = W.mixed_width_primes(70)
    ins, es, s = inputs(W.SEED_BASE + 950, n_ct, moduli, N)
    plan = capi.Plan(N, moduli)
    fwd, inv = step_schedules(14, 7, 1)
    plan.set_schedule(fwd, plan.FORWARD)
    plan.set_schedule(inv, plan.INVERSE)
    got, launches = run(plan, ins, es, s, n_ct, in_place=True)
    assert launches == 4
    for g, e in zip(got, expected(ins, es, s, moduli)):
        np.testing.assert_array_equal(g, e)


def test_fallback_when_row_passes_differ(hexlib):
    """Forward and inverse row passes over different stages: the call runs
    the forward transform and the fused inverse instead, same bits."""
    N, n_ct = 1 << 15, 2
    moduli = W.mixed_width_primes(5)
    ins, es, s = inputs(W.SEED_BASE + 960, n_ct, moduli, N)
    plan = capi.Plan(N, moduli)
    plan.set_schedule([(0, 7, 0, 4, 4, 0, 1), (7, 8, 1, 0, 3, 0, 1)], plan.FORWARD)
    plan.set_schedule([(0, 8, 0, 4, 4, 0, 1), (8, 7, 1, 0, 3, 0, 2)], plan.INVERSE)
    got, launches = run(plan, ins, es, s, n_ct)
    assert launches == 4                      # forward: 2, fused inverse: 2
    for g, e in zip(got, expected(ins, es, s, moduli)):
        np.testing.assert_array_equal(g, e)


HX_ERR_MODULUS, HX_ERR_ARG, HX_ERR_OVERLAP = -4, -8, -9   # include/hexgpu.h


def test_rejects_bad_arguments(hexlib):
    import torch
    N, n_ct = 1 << 12, 1
    moduli = W.mixed_width_primes(3)
    plan = capi.Plan(N, moduli)
    ins, es, s = inputs(W.SEED_BASE + 970, n_ct, moduli, N)
    d_in, d_e = to_device(ins), to_device(es)
    R, work = empty((3,) + ins.shape[1:]), empty(ins.shape)
    with pytest.raises(capi.HexError) as ei:          # result overlapping the inputs
        capi.hx_ciphertext_step(plan, d_in[:3], d_in, work, s, d_e, n_ct)
    assert ei.value.status == HX_ERR_OVERLAP
    with pytest.raises(capi.HexError) as ei:          # a scalar not below its modulus
        capi.hx_ciphertext_step(plan, R, d_in, work, [moduli[0]] + list(s[1:]), d_e, n_ct)
    assert ei.value.status == HX_ERR_ARG
    with pytest.raises(capi.HexError) as ei:
        capi.hx_ciphertext_step(plan, R, d_in, work, s, d_e, 0)
    assert ei.value.status == HX_ERR_ARG
    big = capi.Plan(N, W.mixed_width_primes(1, widths=(62, 62, 62)))
    R1, w1 = empty((3, n_ct, 1, N)), empty((4, n_ct, 1, N))
    i1, e1 = empty((4, n_ct, 1, N)), empty((3, n_ct, 1, N))
    with pytest.raises(capi.HexError) as ei:          # moduli must be below 2^61
        capi.hx_ciphertext_step(big, R1, i1, w1, [1], e1, n_ct)
    assert ei.value.status == HX_ERR_MODULUS
    torch.cuda.synchronize()
