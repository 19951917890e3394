"""The ragged kernels under every column/row split of their menu (the knob
the ragged autotuner turns): for each N from 2^12 to 2^17 and each split,
a ragged set of transforms (limbs of every word path) forward through
hx_ntt_ragged and a batch, inverse back, and a ragged product -- every
output compared element by element with the oracle; the 512-polynomial
ragged workload fully checked under the tuner's choice; the split setting
is validated and restored."""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
import workloads as W
from paper_2103_16400_gb300 import capi, tune
from paper_2103_16400_gb300.tensors import empty, to_device, to_host

pytestmark = pytest.mark.gpu

WIDE4 = W.mixed_width_primes(4, widths=(30, 50, 60, 62))
DEFAULT = {12: 5, 13: 6, 14: 7, 15: 7, 16: 8, 17: 8}


@pytest.fixture
def restore_splits(hexlib):
    keep = {L: capi.hx_ragged_get_split(L) for L in range(12, 18)}
    yield
    for L, k in keep.items():
        capi.hx_ragged_set_split(L, k)


def test_split_setting_is_checked(restore_splits):
    assert {L: capi.hx_ragged_get_split(L) for L in range(12, 18)} == DEFAULT
    assert [tune.ragged_splits(L) for L in (11, 12, 16, 17)] == [[], [5, 6], [5, 6, 7, 8, 9],
                                                                 [6, 7, 8, 9]]
    for L, k in ((12, 7), (16, 4), (17, 5), (11, 5), (18, 9)):
        with pytest.raises(capi.HexError) as e:
            capi.hx_ragged_set_split(L, k)
        assert e.value.status == -8
    capi.hx_ragged_set_split(16, 9)
    assert capi.hx_ragged_get_split(16) == 9


@pytest.mark.parametrize("logN", range(12, 18))
def test_every_split_bit_exact(restore_splits, logN):
    import torch
    N = 1 << logN
    x = W.poly_batch(W.SEED_BASE + 1300 + logN, 0, 2, WIDE4, N)
    exp = oracle.ntt_forward(x, WIDE4)
    plan = capi.Plan(N, WIDE4)
    qs3 = W.mixed_width_primes(3)                      # the product: moduli below 2^61
    a = W.poly_batch(W.SEED_BASE + 1300 + logN, 1, 1, qs3, N)
    b = W.poly_batch(W.SEED_BASE + 1300 + logN, 2, 1, qs3, N)
    prod = oracle.poly_mul(a, b, qs3)
    pplan = capi.Plan(N, qs3)
    for k1 in tune.ragged_splits(logN):
        capi.hx_ragged_set_split(logN, k1)
        dx, dy = to_device(x), empty(x.shape)
        items = [(plan, dx, dy, 2)]
        wsb = capi.hx_ntt_ragged_workspace(items)
        ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
        capi.hx_ntt_ragged(items, ws, wsb, 1, 1, 1)
        if not np.array_equal(to_host(dy), exp):
            pytest.fail(f"forward differs at N=2^{logN}, k1={k1}")
        capi.hx_ntt_ragged([(plan, dy, dy, 2)], ws, wsb, 2, 1, 1)
        if not np.array_equal(to_host(dy), x):
            pytest.fail(f"inverse differs at N=2^{logN}, k1={k1}")
        dz = empty(x.shape)
        capi.Batch([(plan, dx, dz, 2)], 1, 1, 1).run()
        torch.cuda.synchronize()
        if not np.array_equal(to_host(dz), exp):
            pytest.fail(f"batch forward differs at N=2^{logN}, k1={k1}")
        da, db, dr = to_device(a), to_device(b), empty(a.shape)
        pit = [(pplan, da, db, dr, 1)]
        pwsb = capi.hx_polymul_ragged_workspace(pit)
        pws = torch.empty(pwsb, dtype=torch.uint8, device="cuda")
        capi.hx_polymul_ragged(pit, pws, pwsb)
        if not np.array_equal(to_host(dr), prod):
            pytest.fail(f"ragged product differs at N=2^{logN}, k1={k1}")


def test_tuned_512_polynomial_workload_fully_checked(restore_splits, tmp_path, monkeypatch):
    """The bench's ragged workload under the tuner's splits: every one of
    its forward transforms against the oracle (threads over the items; the
    oracle's C calls release the interpreter lock), and the inverse back."""
    import torch
    monkeypatch.setattr(tune, "CACHE_PATH", str(tmp_path / "cache.json"))
    entries = W.ragged_batch(512)
    plans, hosts, dins, douts = [], [], [], []
    for k, (N, qs) in enumerate(entries):
        x = W.poly_batch(W.SEED_BASE + 4, k, 1, qs, N)
        plans.append(capi.Plan(N, qs))
        hosts.append(x)
        dins.append(to_device(x))
        douts.append(empty(x.shape))
    picked = tune.tune_ragged([(p, i, o, 1) for p, i, o in zip(plans, dins, douts)], reps=1)
    assert sorted(picked) == [L for L in range(12, 18) if any(N == 1 << L for N, _ in entries)]
    for L, r in picked.items():
        assert capi.hx_ragged_get_split(L) == r["k1"] and r["tried"] == len(tune.ragged_splits(L))
    fwd = capi.Batch([(p, i, o, 1) for p, i, o in zip(plans, dins, douts)], 1, 1, 1)
    inv = capi.Batch([(p, o, o, 1) for p, o in zip(plans, douts)], 2, 1, 1)
    fwd.run()
    torch.cuda.synchronize()
    got = [to_host(o) for o in douts]
    with ThreadPoolExecutor(16) as ex:
        exps = list(ex.map(lambda k: oracle.ntt_forward(hosts[k], entries[k][1]),
                           range(len(entries))))
    for k in range(len(entries)):
        np.testing.assert_array_equal(got[k], exps[k])
    inv.run()
    torch.cuda.synchronize()
    for k in range(len(entries)):
        np.testing.assert_array_equal(to_host(douts[k]), hosts[k])
