"""hx_polymul_ragged: a mixed set of negacyclic products (every N from 2^10
to 2^17, different modulus sets, several polynomials per item, results
aliasing an operand or not) in one four-kernel call equals the oracle; the
operands are left untouched; a short workspace is refused."""
import numpy as np
import pytest

import oracle
import workloads as W
from paper_2103_16400_gb300 import capi
from paper_2103_16400_gb300.tensors import empty, to_device, to_host

pytestmark = pytest.mark.gpu

SPEC = [(1 << 10, 3, 2), (1 << 11, 2, 1), (1 << 12, 4, 1), (1 << 13, 2, 2), (1 << 14, 3, 1),
        (1 << 15, 1, 1), (1 << 16, 3, 1), (1 << 17, 2, 1)]


def test_mixed_products_vs_oracle(hexlib):
    import torch
    cases, items = [], []
    for k, (N, nl, P) in enumerate(SPEC):
        qs = W.mixed_width_primes(nl + k % 2)[k % 2:]
        a = W.poly_batch(W.SEED_BASE + 6000, 2 * k, P, qs, N)
        b = W.poly_batch(W.SEED_BASE + 6000, 2 * k + 1, P, qs, N)
        da, db = to_device(a), to_device(b)
        out = da if k % 3 == 0 else empty(a.shape)          # some results overwrite a
        plan = capi.Plan(N, qs)
        cases.append((qs, a, b, da, db, out, k % 3 == 0))
        items.append((plan, da, db, out, P))
    wsb = capi.hx_polymul_ragged_workspace(items)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    capi.hx_polymul_ragged(items, ws, wsb)
    torch.cuda.synchronize()
    for qs, a, b, da, db, out, alias in cases:
        np.testing.assert_array_equal(to_host(out), oracle.poly_mul(a, b, qs))
        np.testing.assert_array_equal(to_host(db), b)
        if not alias:
            np.testing.assert_array_equal(to_host(da), a)
    # a second call reusing the workspace on the same stream
    qs, a, b = cases[-1][0], cases[-1][1], cases[-1][2]
    plan, da2, db2 = items[-1][0], to_device(b), to_device(a)
    out2 = empty(a.shape)
    wsb2 = capi.hx_polymul_ragged_workspace([(plan, da2, db2, out2, 1)])
    capi.hx_polymul_ragged([(plan, da2, db2, out2, 1)], ws, wsb2)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(to_host(out2), oracle.poly_mul(b, a, qs))


def test_short_workspace_and_bad_moduli_are_refused(hexlib):
    import torch
    N, qs = 1 << 12, W.mixed_width_primes(2)
    plan = capi.Plan(N, qs)
    a = empty((1, 2, N))
    wsb = capi.hx_polymul_ragged_workspace([(plan, a, a, a, 1)])
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    with pytest.raises(capi.HexError) as e:
        capi.hx_polymul_ragged([(plan, a, a, a, 1)], ws, wsb - 1)
    assert e.value.status == -12
    big = capi.Plan(N, list(W.ntt_primes(62, 2 * N, 1)))        # 4q >= 2^63
    b = empty((1, 1, N))
    with pytest.raises(capi.HexError) as e:
        capi.hx_polymul_ragged_workspace([(big, b, b, b, 1)])
    assert e.value.status == -4
