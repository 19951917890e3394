"""Every kernel schedule the autotuner may pick gives the same bits: the
forward and inverse transforms are compared with the oracle under schedules
that between them use every valid pass configuration (pass split, tile
shape, elements per thread, per-tile / persistent double-buffered / staged-
twiddle kernel, polynomials per thread), at N = 2^12 (single and split
passes), 2^14, 2^16 and 2^17, with one limb of each width and two
polynomials."""
import numpy as np
import pytest

import oracle
import workloads as W
from paper_2103_16400_gb300 import capi, tune
from paper_2103_16400_gb300.tensors import empty, to_device, to_host

pytestmark = pytest.mark.gpu

MIXED3 = W.mixed_width_primes(3)


@pytest.mark.parametrize("logN", [12, 14, 16, 17])
def test_all_schedules_bit_exact(hexlib, logN):
    N = 1 << logN
    x = W.poly_batch(W.SEED_BASE + 900 + logN, 1, 2, MIXED3, N)
    fwd_exp = oracle.ntt_forward(x, MIXED3)
    plan = capi.Plan(N, MIXED3)
    dx, dy = to_device(x), empty(x.shape)
    dz = empty(x.shape)
    n_valid = 0
    for sched in tune.covering(plan):
        plan.set_schedule(sched)
        n_valid += 1
        capi.hx_ntt_forward(plan, dy, dx, 2, 1, 1)
        capi.hx_ntt_inverse(plan, dz, dy, 2, 1, 1)
        got = to_host(dy)
        if not np.array_equal(got, fwd_exp):
            pytest.fail(f"forward differs under schedule {sched}")
        if not np.array_equal(to_host(dz), x):
            pytest.fail(f"inverse differs under schedule {sched}")
    assert n_valid >= 4


def test_tuner_picks_a_valid_schedule_and_caches(hexlib, tmp_path, monkeypatch):
    monkeypatch.setattr(tune, "CACHE_PATH", str(tmp_path / "cache.json"))
    N = 1 << 14
    plan = capi.Plan(N, MIXED3)
    res = tune.tune(plan, 2, iters=1)
    assert res["tried"] >= 4 and res["fwd_us"] > 0
    assert [list(p) for p in plan.schedule(plan.FORWARD)] == res["forward"]
    assert [list(p) for p in plan.schedule(plan.INVERSE)] == res["inverse"]
    again = tune.tune(capi.Plan(N, MIXED3), 2)
    assert again.get("cached") and again["forward"] == res["forward"]
    x = W.poly_batch(W.SEED_BASE + 950, 1, 2, MIXED3, N)
    dy = empty(x.shape)
    capi.hx_ntt_forward(plan, dy, to_device(x), 2, 1, 1)
    np.testing.assert_array_equal(to_host(dy), oracle.ntt_forward(x, MIXED3))


def test_tuning_one_direction_keeps_the_other(hexlib, tmp_path, monkeypatch):
    """tune(direction=forward) and tune_tensor (inverse only) each set only
    their own schedule, whether they time candidates or hit the cache."""
    monkeypatch.setattr(tune, "CACHE_PATH", str(tmp_path / "cache.json"))
    N = 1 << 12
    s = W.scalars(W.SEED_BASE + 960, 20, MIXED3)
    for _ in range(2):                                   # timed, then cached
        plan = capi.Plan(N, MIXED3)
        f = tune.tune(plan, 4, iters=1, direction=plan.FORWARD)["forward"]
        inv = tune.tune_tensor(plan, 1, s, iters=1)["inverse"]
        assert [list(p) for p in plan.schedule(plan.FORWARD)] == f
        assert [list(p) for p in plan.schedule(plan.INVERSE)] == inv


def test_launch_order_many_mixed_limbs(hexlib):
    """70 limbs of four widths (30-bit words, truncated- and exact-quotient
    64-bit words): column passes launch them costliest first within runs of
    64; under each covering schedule every limb must still be transformed
    exactly once, bit-exact."""
    N = 1 << 14
    moduli = W.mixed_width_primes(70, widths=(30, 50, 60, 62))
    x = W.poly_batch(W.SEED_BASE + 960, 1, 2, moduli, N)
    fwd_exp = oracle.ntt_forward(x, moduli)
    plan = capi.Plan(N, moduli)
    dx, dy, dz = to_device(x), empty(x.shape), empty(x.shape)
    n = 0
    for sched in tune.covering(plan):
        plan.set_schedule(sched)
        dy.fill_(0)
        dz.fill_(0)
        capi.hx_ntt_forward(plan, dy, dx, 2, 1, 1)
        capi.hx_ntt_inverse(plan, dz, dy, 2, 1, 1)
        if not np.array_equal(to_host(dy), fwd_exp):
            pytest.fail(f"forward differs under schedule {sched}")
        if not np.array_equal(to_host(dz), x):
            pytest.fail(f"inverse differs under schedule {sched}")
        n += 1
    assert n >= 4
