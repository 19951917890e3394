"""Ragged batches (hx_batch_*): transforms of every N from 2^10 to 2^17 and
different modulus sets in one graph replay, compared with the oracle; graph
replays re-arm their work counters; and the 512-polynomial ragged workload
(N ~ U{2^10..2^17}, 1-32 limbs of 30/50/60 bits) round-trips exactly, with
sampled transforms checked against the oracle."""
import numpy as np
import pytest

import oracle
import workloads as W
from paper_2103_16400_gb300 import capi
from paper_2103_16400_gb300.tensors import empty, to_device, to_host

pytestmark = pytest.mark.gpu


def _items(seed, spec):
    """spec: list of (N, moduli, n_polys); returns host arrays and plans."""
    out = []
    for k, (N, qs, P) in enumerate(spec):
        x = W.poly_batch(seed, k, P, qs, N)
        out.append((capi.Plan(N, qs), x))
    return out


SPEC = [(1 << 10, W.mixed_width_primes(2), 3), (1 << 11, W.mixed_width_primes(4), 1),
        (1 << 12, W.mixed_width_primes(3), 2), (1 << 13, W.mixed_width_primes(1), 1),
        (1 << 14, W.mixed_width_primes(5), 1), (1 << 15, W.mixed_width_primes(3)[1:], 2),
        (1 << 16, W.mixed_width_primes(3), 1), (1 << 17, W.mixed_width_primes(2), 1)]


@pytest.mark.parametrize("inplace", [False, True])
def test_ragged_forward_inverse_vs_oracle(hexlib, inplace):
    import torch
    items = _items(W.SEED_BASE + 4000, SPEC)
    dins = [to_device(x) for _, x in items]
    douts = dins if inplace else [empty(x.shape) for _, x in items]
    fwd = capi.Batch([(p, i, o, x.shape[0]) for (p, x), i, o in zip(items, dins, douts)], 1, 1, 1)
    info = fwd.info()
    assert info["limb_transforms"] == sum(x.shape[0] * x.shape[1] for _, x in items)
    fwd.run()
    torch.cuda.synchronize()
    for (p, x), o in zip(items, douts):
        np.testing.assert_array_equal(to_host(o), oracle.ntt_forward(x, p.moduli))
    backs = [empty(x.shape) for _, x in items]
    inv = capi.Batch([(p, o, b, x.shape[0]) for (p, x), o, b in zip(items, douts, backs)], 2, 1, 1)
    inv.run()
    torch.cuda.synchronize()
    for (p, x), b in zip(items, backs):
        np.testing.assert_array_equal(to_host(b), x)


def test_ragged_replay_and_lazy_ranges(hexlib):
    """Three replays of the same graph (counters re-armed each time), lazy
    output range 4 for the forward and 2 for the inverse."""
    import torch
    spec = SPEC[::2]
    items = _items(W.SEED_BASE + 4100, spec)
    dins = [to_device(x) for _, x in items]
    douts = [empty(x.shape) for _, x in items]
    fwd = capi.Batch([(p, i, o, x.shape[0]) for (p, x), i, o in zip(items, dins, douts)], 1, 1, 4)
    for _ in range(3):
        fwd.run()
    torch.cuda.synchronize()
    for (p, x), o in zip(items, douts):
        got = to_host(o)
        exp = oracle.ntt_forward(x, p.moduli)
        for l, q in enumerate(p.moduli):
            assert (got[:, l] < np.uint64(4 * q)).all()
            np.testing.assert_array_equal(got[:, l] % np.uint64(q), exp[:, l])
    # inverse inputs in [0, 2q): the canonical spectra lifted by 0 or q
    specs = []
    for k, (p, x) in enumerate(items):
        y = oracle.ntt_forward(x, p.moduli)
        for l, q in enumerate(p.moduli):
            y[:, l] = W.lazy_lift(100 + 7 * k + l, y[:, l].reshape(-1), q, 2).reshape(y[:, l].shape)
        specs.append(to_device(y))
    inv = capi.Batch([(p, s, s, x.shape[0]) for (p, x), s in zip(items, specs)], 2, 2, 2)
    inv.run()
    torch.cuda.synchronize()
    for (p, x), o in zip(items, specs):
        got = to_host(o)
        for l, q in enumerate(p.moduli):
            assert (got[:, l] < np.uint64(2 * q)).all()
            np.testing.assert_array_equal(got[:, l] % np.uint64(q), x[:, l])


def test_ragged_batch_argument_errors(hexlib):
    p = capi.Plan(1 << 10, W.mixed_width_primes(1))
    buf = empty((1, 1, 1 << 10))
    with pytest.raises(capi.HexError) as e:
        capi.Batch([(p, buf, buf, 1)], 1, 1, 2)          # forward out_mf 2
    assert e.value.status == -6
    with pytest.raises(capi.HexError) as e:
        capi.Batch([(p, buf.data_ptr() + 8, buf, 1)], 1, 1, 1)
    assert e.value.status == -2
    with pytest.raises(capi.HexError) as e:
        capi.Batch([(p, buf, buf, 1)], 3, 1, 1)           # bad direction
    assert e.value.status == -8


def test_ragged_512_polynomial_workload(hexlib):
    import torch
    entries = W.ragged_batch(512)
    plans, hosts, dins, douts = [], [], [], []
    for k, (N, qs) in enumerate(entries):
        x = W.poly_batch(W.SEED_BASE + 4, k, 1, qs, N)
        plans.append(capi.Plan(N, qs))
        hosts.append(x)
        dins.append(to_device(x))
        douts.append(empty(x.shape))
    fwd = capi.Batch([(p, i, o, 1) for p, i, o in zip(plans, dins, douts)], 1, 1, 1)
    inv = capi.Batch([(p, o, o, 1) for p, o in zip(plans, douts)], 2, 1, 1)
    fwd.run()
    torch.cuda.synchronize()
    rng = np.random.default_rng(7)
    for k in rng.choice(len(entries), 24, replace=False):     # sampled oracle checks
        N, qs = entries[k]
        l = int(rng.integers(len(qs)))
        np.testing.assert_array_equal(to_host(douts[k])[0, l],
                                      oracle.ntt_forward_1(hosts[k][0, l], qs[l]))
    inv.run()
    torch.cuda.synchronize()
    for k in range(len(entries)):                              # every transform round-trips
        np.testing.assert_array_equal(to_host(douts[k]), hosts[k])


def test_plans_share_twiddle_tables(hexlib):
    """Plans over overlapping (N, q) share one table; destroying one plan
    leaves the other's tables alive and its results exact."""
    qs = W.mixed_width_primes(4)
    N = 1 << 12
    p1 = capi.Plan(N, qs[:3])
    p2 = capi.Plan(N, qs[1:])
    b1 = p1.info()[2]
    assert b1 >= 3 * 32 * N
    x = W.poly_batch(W.SEED_BASE + 4200, 0, 1, qs[1:], N)
    p1.destroy()
    y = empty(x.shape)
    capi.hx_ntt_forward(p2, y, to_device(x), 1, 1, 1)
    np.testing.assert_array_equal(to_host(y), oracle.ntt_forward(x, qs[1:]))
