"""hx_tensor_fma_inverse (the ciphertext tensor's element-wise step fused into
the first pass of the inverse transform) against the oracle's composition:
d0 = A0 B0, d1 = A0 B1 + A1 B0, d2 = A1 B1, r_k = d_k s + e_k, out_k =
InvNTT(r_k).  Covers single- and two-pass schedules, every schedule whose
first inverse pass can carry the fusion, more limbs than one launch holds,
lazy inputs (input_mod_factor 2 and 4), and the unfused fallbacks
(operands not back to back; a persistent first pass) -- all must give the
same bits."""
import numpy as np
import pytest

import oracle
import workloads as W
from paper_2103_16400_gb300 import capi, tune
from paper_2103_16400_gb300.tensors import empty, to_device, to_host

pytestmark = pytest.mark.gpu


def expected(A, E, s, moduli):
    """A: [4][n][L][N] forward outputs (any representative), E: [3][n][L][N]."""
    Ar = [np.stack([A[i][:, l] % np.uint64(q) for l, q in enumerate(moduli)], axis=1)
          for i in range(4)]
    d0 = oracle.eltwise_mult_mod(Ar[0], Ar[2], moduli)
    d1 = oracle.eltwise_add_mod(oracle.eltwise_mult_mod(Ar[0], Ar[3], moduli),
                                oracle.eltwise_mult_mod(Ar[1], Ar[2], moduli), moduli)
    d2 = oracle.eltwise_mult_mod(Ar[1], Ar[3], moduli)
    return [oracle.ntt_inverse(oracle.eltwise_fma_mod(d, s, e, moduli), moduli)
            for d, e in ((d0, E[0]), (d1, E[1]), (d2, E[2]))]


def operands(seed, n_ct, moduli, N, in_mf):
    A = np.stack([W.poly_batch(seed, t, n_ct, moduli, N) for t in range(4)])
    if in_mf > 1:
        for t in range(4):
            for p in range(n_ct):
                for l, q in enumerate(moduli):
                    key = W.stream_key(seed, 50 + t, p, l)
                    A[t, p, l] = W.lazy_lift(key, A[t, p, l], q, in_mf)
    E = np.stack([W.poly_batch(seed, 10 + t, n_ct, moduli, N) for t in range(3)])
    s = W.scalars(seed, 20, moduli)
    return A, E, s


def run_fused(plan, A, E, s, n_ct, in_mf):
    dA, dE = to_device(A), to_device(E)
    R = empty((3,) + A.shape[1:])
    capi.hx_tensor_fma_inverse(plan, R[0], R[1], R[2], dA[0], dA[1], dA[2], dA[3], s,
                               dE[0], dE[1], dE[2], n_ct, in_mf)
    return [to_host(R[k]) for k in range(3)]


@pytest.mark.parametrize("logN,n_limbs,n_ct,in_mf", [(10, 3, 2, 4), (12, 4, 1, 1),
                                                     (14, 6, 2, 2), (16, 5, 1, 4)])
def test_fused_matches_oracle(hexlib, logN, n_limbs, n_ct, in_mf):
    N = 1 << logN
    moduli = W.mixed_width_primes(n_limbs)
    A, E, s = operands(W.SEED_BASE + 700 + logN, n_ct, moduli, N, in_mf)
    plan = capi.Plan(N, moduli)
    exp = expected(A, E, s, moduli)
    for got, e in zip(run_fused(plan, A, E, s, n_ct, in_mf), exp):
        np.testing.assert_array_equal(got, e)


def test_every_fusable_schedule(hexlib):
    """All schedules of the covering set at N = 2^13 and 2^14 (per-tile and
    staged-twiddle first passes fuse; persistent ones take the fallback)."""
    for logN in (13, 14):
        N = 1 << logN
        moduli = W.mixed_width_primes(3)
        A, E, s = operands(W.SEED_BASE + 740 + logN, 1, moduli, N, 4)
        exp = expected(A, E, s, moduli)
        plan = capi.Plan(N, moduli)
        n = 0
        for sched in tune.covering(plan):
            plan.set_schedule(sched)
            for got, e in zip(run_fused(plan, A, E, s, 1, 4), exp):
                if not np.array_equal(got, e):
                    pytest.fail(f"differs under schedule {sched}")
            n += 1
        assert n >= 8


def test_more_limbs_than_one_launch(hexlib):
    N = 1 << 11
    moduli = W.mixed_width_primes(70)
    A, E, s = operands(W.SEED_BASE + 760, 1, moduli, N, 2)
    plan = capi.Plan(N, moduli)
    for got, e in zip(run_fused(plan, A, E, s, 1, 2), expected(A, E, s, moduli)):
        np.testing.assert_array_equal(got, e)


def test_unfused_layouts_give_the_same_bits(hexlib):
    N = 1 << 12
    moduli = W.mixed_width_primes(3)
    A, E, s = operands(W.SEED_BASE + 770, 2, moduli, N, 4)
    exp = expected(A, E, s, moduli)
    plan = capi.Plan(N, moduli)
    # separate buffers: no back-to-back layout
    dA = [to_device(A[i]) for i in range(4)]
    dE = [to_device(E[i]) for i in range(3)]
    R = [empty(A.shape[1:]) for _ in range(3)]
    capi.hx_tensor_fma_inverse(plan, R[0], R[1], R[2], *dA, s, *dE, 2, 4)
    for r, e in zip(R, exp):
        np.testing.assert_array_equal(to_host(r), e)
    # a persistent first inverse pass: the composed path
    plan.set_schedule([(0, 6, 0, 3, 3, 0, 1), (6, 6, 2, 0, 3, 1, 1)])
    for got, e in zip(run_fused(plan, A, E, s, 2, 4), exp):
        np.testing.assert_array_equal(got, e)


def test_rejects_bad_arguments(hexlib):
    N = 1 << 10
    moduli = W.mixed_width_primes(2)
    plan = capi.Plan(N, moduli)
    A = empty((4, 1, 2, N))
    E = empty((3, 1, 2, N))
    s = W.scalars(W.SEED_BASE + 780, 20, moduli)
    with pytest.raises(capi.HexError):          # output overlapping an input
        capi.hx_tensor_fma_inverse(plan, A[0], A[1], A[2], A[0], A[1], A[2], A[3], s,
                                   E[0], E[1], E[2], 1, 4)
    R = empty((3, 1, 2, N))
    with pytest.raises(capi.HexError):          # bad input_mod_factor
        capi.hx_tensor_fma_inverse(plan, R[0], R[1], R[2], A[0], A[1], A[2], A[3], s,
                                   E[0], E[1], E[2], 1, 3)
    bad = np.array([moduli[0], moduli[1] + 1], dtype=np.uint64)
    with pytest.raises(capi.HexError):          # scalar >= q
        capi.hx_tensor_fma_inverse(plan, R[0], R[1], R[2], A[0], A[1], A[2], A[3], bad,
                                   E[0], E[1], E[2], 1, 4)


def test_launch_order_two_pass_many_limbs(hexlib):
    """Two-pass schedules at N = 2^14 with 70 limbs of the 30/50/60-bit mix
    (the tensor's FMA takes moduli below 2^61): the fused pass (two launches
    of up to 64 limbs) and the column pass both take the 64-bit-word limbs
    first; every result must be the oracle's."""
    N = 1 << 14
    moduli = W.mixed_width_primes(70)
    A, E, s = operands(W.SEED_BASE + 790, 1, moduli, N, 4)
    exp = expected(A, E, s, moduli)
    plan = capi.Plan(N, moduli)
    scheds = [sc for sc in tune.covering(plan) if len(sc) == 2][:6]
    assert scheds
    for sched in scheds:
        plan.set_schedule(sched)
        for got, e in zip(run_fused(plan, A, E, s, 1, 4), exp):
            if not np.array_equal(got, e):
                pytest.fail(f"differs under schedule {sched}")
