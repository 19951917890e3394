"""hx_poly_mul with the dyadic product computed in the inverse's first pass:
the same bits as the oracle's product (fwd, fwd, MultMod, inv -- Listing 4)
under every schedule of the covering set, whether that pass can carry the
product (per-tile row or single pass) or not (persistent first pass,
cluster-fused schedules: the separate element-wise pass), for limbs of every
word path (30-bit words, truncated- and exact-quotient 64-bit words), with
the result aliasing an operand; and one kernel launch fewer when fused."""
import numpy as np
import pytest

import oracle
import workloads as W
from paper_2103_16400_gb300 import capi, tune
from paper_2103_16400_gb300.tensors import empty, to_device, to_host

pytestmark = pytest.mark.gpu

WIDE4 = W.mixed_width_primes(4, widths=(30, 50, 60, 62))


@pytest.mark.parametrize("logN", [12, 14, 16])
def test_product_under_every_schedule(hexlib, logN):
    N = 1 << logN
    a = W.poly_batch(W.SEED_BASE + 1200 + logN, 0, 2, WIDE4, N)
    b = W.poly_batch(W.SEED_BASE + 1200 + logN, 1, 2, WIDE4, N)
    exp = oracle.poly_mul(a, b, WIDE4)
    if logN == 12:                     # the oracle's product against the schoolbook
        for l, q in enumerate(WIDE4):
            np.testing.assert_array_equal(exp[1, l], oracle.negacyclic_schoolbook(a[1, l],
                                                                                   b[1, l], q))
    plan = capi.Plan(N, WIDE4)
    scheds = tune.covering(plan)
    if logN == 16:
        scheds = scheds[::4]
    n_fused = 0
    for sched in scheds:
        plan.set_schedule(sched)
        last = sched[-1]
        n_fused += last[5] in (0, 2) and (len(sched) == 1 or last[3] == 0)
        da, db, r = to_device(a), to_device(b), empty(a.shape)
        capi.hx_poly_mul(plan, r, da, db, 2)
        if not np.array_equal(to_host(r), exp):
            pytest.fail(f"product differs under schedule {sched}")
        da, db = to_device(a), to_device(b)
        capi.hx_poly_mul(plan, da, da, db, 2)            # result overwrites a
        if not np.array_equal(to_host(da), exp):
            pytest.fail(f"in-place product differs under schedule {sched}")
    assert n_fused >= 2


def test_fused_product_saves_a_launch(hexlib):
    import torch
    N = 1 << 14
    plan = capi.Plan(N, WIDE4)
    a = W.poly_batch(W.SEED_BASE + 1230, 0, 1, WIDE4, N)
    b = W.poly_batch(W.SEED_BASE + 1230, 1, 1, WIDE4, N)
    exp = oracle.poly_mul(a, b, WIDE4)
    counts = {}
    for name, sched in (("fused", [(0, 7, 0, 3, 4, 0, 1), (7, 7, 1, 0, 3, 0, 1)]),
                        ("composed", [(0, 7, 0, 3, 4, 0, 1), (7, 7, 1, 0, 3, 1, 1)])):
        plan.set_schedule(sched)
        da, db, r = to_device(a), to_device(b), empty(a.shape)
        torch.cuda.synchronize()
        n0 = capi.hx_launch_count()
        capi.hx_poly_mul(plan, r, da, db, 1)
        counts[name] = capi.hx_launch_count() - n0
        np.testing.assert_array_equal(to_host(r), exp)
    # two forward calls of two passes, then the inverse's two passes (with
    # the product inside the first) -- or the element-wise kernel on top
    assert counts == {"fused": 6, "composed": 7}


@pytest.mark.parametrize("logN", [12, 14])
def test_dyadic_inverse(hexlib, logN):
    """hx_dyadic_inverse(A, B) = InvNTT(A . B) for spectra below 4q (lifted
    by k q), fused (row-pass first inverse pass) and composed (persistent
    first pass), into a fresh buffer and onto A itself; A and B untouched
    otherwise."""
    N = 1 << logN
    qs = W.mixed_width_primes(4, widths=(30, 50, 60, 62))
    seed = W.SEED_BASE + 1240 + logN
    a = W.poly_batch(seed, 0, 2, qs, N)
    b = W.poly_batch(seed, 1, 2, qs, N)
    exp = oracle.poly_mul(a, b, qs)
    A, B = oracle.ntt_forward(a, qs), oracle.ntt_forward(b, qs)
    for p in range(2):
        for l, q in enumerate(qs):
            A[p, l] = W.lazy_lift(W.stream_key(seed, 5, p, l), A[p, l], q, 4)
            B[p, l] = W.lazy_lift(W.stream_key(seed, 6, p, l), B[p, l], q, 4)
    plan = capi.Plan(N, qs)
    K1, gb = logN // 2, 2 if logN == 12 else 1         # row tiles of 32 threads or more
    for sched in ([(0, K1, 0, 3, 4, 0, 1), (K1, logN - K1, gb, 0, 3, 0, 1)],
                  [(0, K1, 0, 3, 4, 0, 1), (K1, logN - K1, gb, 0, 3, 1, 1)]):
        plan.set_schedule(sched)
        dA, dB, r = to_device(A), to_device(B), empty(A.shape)
        capi.hx_dyadic_inverse(plan, r, dA, dB, 2, 4)
        np.testing.assert_array_equal(to_host(r), exp)
        np.testing.assert_array_equal(to_host(dA), A)
        np.testing.assert_array_equal(to_host(dB), B)
        capi.hx_dyadic_inverse(plan, dA, dA, dB, 2, 4)
        np.testing.assert_array_equal(to_host(dA), exp)
    with pytest.raises(capi.HexError):
        capi.hx_dyadic_inverse(plan, r, dA, dB, 2, 8)        # input_mod_factor 8
