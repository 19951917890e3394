"""The cluster-fused transform (one thread-block cluster per limb-transform,
every stage in shared memory, the column/row exchange through distributed
shared memory) against the oracle, element by element: every cluster
schedule the library accepts at N = 2^14 .. 2^17 on limbs of every word
path (30-bit words, truncated- and exact-quotient 64-bit words), lazy input
and output ranges, in-place calls, more limbs than the launch order's runs,
the ciphertext tensor fused into the cluster inverse, and the benchmark's
full size (N = 2^16, 32 limbs, 4 polynomials)."""
import numpy as np
import pytest

import oracle
import workloads as W
from paper_2103_16400_gb300 import capi, tune
from paper_2103_16400_gb300.tensors import empty, to_device, to_host

pytestmark = pytest.mark.gpu

WIDE4 = W.mixed_width_primes(4, widths=(30, 50, 60, 62))


def cluster_scheds(plan):
    logN = plan.N.bit_length() - 1
    return [s for s in tune.cluster_options(logN) if tune.valid(plan, s)]


def check_lazy(got, exp, moduli, mf):
    """out_mf > 1: every value below mf q and congruent to the oracle's."""
    for l, q in enumerate(moduli):
        g = got[:, l]
        assert (g < np.uint64(mf * q)).all()
        np.testing.assert_array_equal(g % np.uint64(q), exp[:, l])


@pytest.mark.parametrize("logN", [14, 15, 16, 17])
def test_every_cluster_schedule_bit_exact(hexlib, logN):
    N = 1 << logN
    x = W.poly_batch(W.SEED_BASE + 1100 + logN, 1, 2, WIDE4, N)
    fwd_exp = oracle.ntt_forward(x, WIDE4)
    plan = capi.Plan(N, WIDE4)
    scheds = cluster_scheds(plan)
    assert len(scheds) >= 3, scheds
    dx, dy, dz = to_device(x), empty(x.shape), empty(x.shape)
    for sched in scheds:
        plan.set_schedule(sched)
        dy.fill_(0)
        dz.fill_(0)
        capi.hx_ntt_forward(plan, dy, dx, 2, 1, 1)
        capi.hx_ntt_inverse(plan, dz, dy, 2, 1, 1)
        if not np.array_equal(to_host(dy), fwd_exp):
            pytest.fail(f"forward differs under schedule {sched}")
        if not np.array_equal(to_host(dz), x):
            pytest.fail(f"inverse differs under schedule {sched}")


@pytest.mark.parametrize("logN", [15, 16])
def test_cluster_lazy_ranges_and_in_place(hexlib, logN):
    N = 1 << logN
    plan = capi.Plan(N, WIDE4)
    seed = W.SEED_BASE + 1120 + logN
    x = W.poly_batch(seed, 1, 2, WIDE4, N)
    fwd_exp = oracle.ntt_forward(x, WIDE4)
    for sched in cluster_scheds(plan)[:4]:
        plan.set_schedule(sched)
        for in_mf in (2, 4):
            xl = x.copy()
            for p in range(2):
                for l, q in enumerate(WIDE4):
                    xl[p, l] = W.lazy_lift(W.stream_key(seed, 7, p, l), x[p, l], q, in_mf)
            d = to_device(xl)
            capi.hx_ntt_forward(plan, d, d, 2, in_mf, 4)           # in place, out in [0, 4q)
            check_lazy(to_host(d), fwd_exp, WIDE4, 4)
        yl = fwd_exp.copy()
        for p in range(2):
            for l, q in enumerate(WIDE4):
                yl[p, l] = W.lazy_lift(W.stream_key(seed, 8, p, l), fwd_exp[p, l], q, 2)
        d = to_device(yl)
        capi.hx_ntt_inverse(plan, d, d, 2, 2, 2)                   # in place, lazy in and out
        check_lazy(to_host(d), x, WIDE4, 2)
        d = to_device(x)
        capi.hx_ntt_forward(plan, d, d, 2, 1, 1)
        np.testing.assert_array_equal(to_host(d), fwd_exp)


def test_cluster_many_limbs_launch_order(hexlib):
    """70 limbs of four widths: the cluster launch takes the limbs in the
    plan's cost order; each must still be transformed once, bit-exact."""
    N = 1 << 14
    moduli = W.mixed_width_primes(70, widths=(30, 50, 60, 62))
    x = W.poly_batch(W.SEED_BASE + 1140, 1, 1, moduli, N)
    fwd_exp = oracle.ntt_forward(x, moduli)
    plan = capi.Plan(N, moduli)
    dx, dy, dz = to_device(x), empty(x.shape), empty(x.shape)
    for sched in cluster_scheds(plan):
        plan.set_schedule(sched)
        capi.hx_ntt_forward(plan, dy, dx, 1, 1, 1)
        capi.hx_ntt_inverse(plan, dz, dy, 1, 1, 1)
        if not np.array_equal(to_host(dy), fwd_exp):
            pytest.fail(f"forward differs under schedule {sched}")
        if not np.array_equal(to_host(dz), x):
            pytest.fail(f"inverse differs under schedule {sched}")


def tensor_expected(A, E, s, moduli):
    Ar = [np.stack([A[i][:, l] % np.uint64(q) for l, q in enumerate(moduli)], axis=1)
          for i in range(4)]
    d0 = oracle.eltwise_mult_mod(Ar[0], Ar[2], moduli)
    d1 = oracle.eltwise_add_mod(oracle.eltwise_mult_mod(Ar[0], Ar[3], moduli),
                                oracle.eltwise_mult_mod(Ar[1], Ar[2], moduli), moduli)
    d2 = oracle.eltwise_mult_mod(Ar[1], Ar[3], moduli)
    return [oracle.ntt_inverse(oracle.eltwise_fma_mod(d, s, e, moduli), moduli)
            for d, e in ((d0, E[0]), (d1, E[1]), (d2, E[2]))]


@pytest.mark.parametrize("logN,n_limbs,n_ct", [(14, 70, 1), (15, 4, 2), (16, 5, 2), (17, 3, 1)])
def test_cluster_tensor_fused(hexlib, logN, n_limbs, n_ct):
    N = 1 << logN
    moduli = W.mixed_width_primes(n_limbs)
    seed = W.SEED_BASE + 1160 + logN
    A = np.stack([W.poly_batch(seed, t, n_ct, moduli, N) for t in range(4)])
    for t in range(4):
        for p in range(n_ct):
            for l, q in enumerate(moduli):
                A[t, p, l] = W.lazy_lift(W.stream_key(seed, 50 + t, p, l), A[t, p, l], q, 4)
    E = np.stack([W.poly_batch(seed, 10 + t, n_ct, moduli, N) for t in range(3)])
    s = W.scalars(seed, 20, moduli)
    exp = tensor_expected(A, E, s, moduli)
    plan = capi.Plan(N, moduli)
    dA, dE = to_device(A), to_device(E)
    R = empty((3,) + A.shape[1:])
    scheds = cluster_scheds(plan)
    assert scheds
    for sched in scheds[:: max(1, len(scheds) // 4)]:
        plan.set_schedule(sched)
        R.fill_(0)
        capi.hx_tensor_fma_inverse(plan, R[0], R[1], R[2], dA[0], dA[1], dA[2], dA[3], s,
                                   dE[0], dE[1], dE[2], n_ct, 4)
        for k in range(3):
            if not np.array_equal(to_host(R[k]), exp[k]):
                pytest.fail(f"tensor output {k} differs under schedule {sched}")


def test_cluster_full_size_forward_inverse(hexlib):
    """N = 2^16 x 32 mixed limbs x 4 polynomials (the benchmark's forward
    call) under each cluster schedule with 16 elements a thread."""
    N, nl = 1 << 16, 32
    moduli = W.mixed_width_primes(nl)
    x = W.poly_batch(W.SEED_BASE + 1180, 1, 4, moduli, N)
    fwd_exp = oracle.ntt_forward(x, moduli)
    plan = capi.Plan(N, moduli)
    dx, dy, dz = to_device(x), empty(x.shape), empty(x.shape)
    n = 0
    for sched in cluster_scheds(plan):
        if sched[0][4] != 4:
            continue
        plan.set_schedule(sched)
        capi.hx_ntt_forward(plan, dy, dx, 4, 1, 1)
        capi.hx_ntt_inverse(plan, dz, dy, 4, 1, 1)
        if not np.array_equal(to_host(dy), fwd_exp):
            pytest.fail(f"forward differs under schedule {sched}")
        if not np.array_equal(to_host(dz), x):
            pytest.fail(f"inverse differs under schedule {sched}")
        n += 1
    assert n >= 2
